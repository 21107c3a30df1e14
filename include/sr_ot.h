/*
 * sr_ot.h -- C ABI of the GB300 (sm_103a) block-coordinate Frank-Wolfe solver
 * for squared-l2 semi-relaxed optimal transport (Fukunaga & Kasai,
 * arXiv 2103.05857).
 *
 * Problem (Sec. 3, eq. 5, stated here in the library's orientation, which is
 * the transpose of the paper's: rows are the blocks):
 *
 *     minimise  f(T) = <C, T> + (rho/2) || T^T 1_m - b ||^2
 *     over      T in R^{m x n}, T >= 0, T 1_n = a          (eq. 6: product of
 *                                                           scaled simplices)
 *
 * rho = 1/lambda of the paper. The block gradient of row i is
 * grad_i = C_{i,:} + rho (s - b), s = T^T 1_m (Sec. 3.1); the linear
 * minimisation oracle is a_i e_{j*}, j* = argmin_j grad_ij (eq. 7); the
 * duality gap is g(T) = sum_i <t_i - a_i e_{j*}, grad_i> (Thm 2, eq. 11).
 *
 * Conventions for every entry point:
 *   - All matrices are dense row-major; all sizes are element counts.
 *   - Pointers named X, Y, C, a, b, T, dX, dY, db, dC are DEVICE pointers on
 *     the handle's device, owned by the caller, and must stay valid until the
 *     call returns. Their element type follows opts->precision: double for
 *     SR_OT_FP64, float for SR_OT_FP32 and SR_OT_FP32_BF16COST.
 *   - Pointers to sr_ot_options, sr_ot_result and per-instance size/offset
 *     arrays are HOST pointers.
 *   - Calls are ordered on the handle's stream and return after the stream
 *     has been synchronised (results are final when the call returns).
 *   - One handle per host thread. A handle owns its device workspace (grown
 *     on demand, freed by sr_ot_destroy) and a pinned result buffer.
 *   - Return value: SR_OT_OK or SR_OT_NOT_CONVERGED on success, a negative
 *     sr_ot_status on error; sr_ot_last_error() then describes it. Nothing
 *     aborts, traps or waits without bound.
 */
#ifndef SR_OT_H
#define SR_OT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sr_ot_ctx *sr_ot_handle;

typedef enum {
    SR_OT_OK = 0,
    SR_OT_NOT_CONVERGED = 1,  /* status, not an error: max_epochs reached before tol */
    SR_OT_EINVAL = -1,        /* invalid argument (sizes, pointers, options, weights) */
    SR_OT_ENOMEM = -2,        /* device workspace allocation failed */
    SR_OT_ECUDA = -3,         /* CUDA runtime error */
    SR_OT_ETIMEOUT = -4,      /* a bounded device wait gave up */
    SR_OT_ENUMERIC = -5,      /* non-finite value met in the inputs or iterates */
    SR_OT_EUNSUPPORTED = -6   /* valid request outside this build's limits */
} sr_ot_status;

/* Direction rule (Alg. 1; Alg. A.2 away steps; Alg. A.3 pairwise steps;
 * Alg. A.1 full FW). */
typedef enum { SR_OT_BCFW = 0, SR_OT_BCAFW = 1, SR_OT_BCPFW = 2, SR_OT_FW = 3 } sr_ot_variant;

/* Block order (Sec. 3.1: U = uniform, P = fresh permutation per epoch;
 * Sec. 4.2 / Alg. A.4: gap-adaptive sampling, "BCFW-GA"). */
typedef enum {
    SR_OT_CYCLIC = 0,
    SR_OT_PERMUTE = 1,
    SR_OT_UNIFORM = 2,
    SR_OT_GAP_ADAPTIVE = 3
} sr_ot_order;

/* Step rule (Alg. 1): decay 2m/(k+2m) (FW: 2/(k+2)) or exact line search
 * (eq. 8; eq. 10 for away/pairwise, which require SR_OT_ELS). */
typedef enum { SR_OT_DEC = 0, SR_OT_ELS = 1 } sr_ot_step;

/* Arithmetic. SR_OT_FP64: everything in double. SR_OT_FP32: float plan,
 * cost and row updates; the duality gap, column-sum refresh and stopping test
 * accumulate in double. SR_OT_FP32_BF16COST: as SR_OT_FP32, with the cost
 * C = |x|^2 + |y|^2 - 2 X Y^T built by a BF16 tensor-core GEMM with FP32
 * accumulation and FP32 norms (points mode, d a multiple of 64). */
typedef enum { SR_OT_FP64 = 0, SR_OT_FP32 = 1, SR_OT_FP32_BF16COST = 2 } sr_ot_precision;

/* Cost built from points (sr_ot_options.cost_kind). */
typedef enum {
    SR_OT_COST_SQUARED = 0,   /* C_ij = ||x_i - y_j||^2                             */
    SR_OT_COST_EUCLIDEAN = 1  /* C_ij = ||x_i - y_j||_2 (the paper's, Sec. 5.1)     */
} sr_ot_cost_kind;

/* Active-set epoch kernels for FP32 pairwise solves (sr_ot_options.epoch_kernel). */
typedef enum {
    SR_OT_EPOCH_AUTO = 0,
    SR_OT_EPOCH_TWO_PHASE = 1,    /* the next row's LMO waits for the current update   */
    SR_OT_EPOCH_PIPELINED = 2,    /* the next row's LMO and away vertex overlap the
                                     current update (two alternating control warps)    */
    SR_OT_EPOCH_SPECULATIVE = 3,  /* LMOs of the next rows taken ahead against an older
                                     residual and repaired at the changed columns;
                                     three chain warps take the updates in turn        */
    SR_OT_EPOCH_SPECULATIVE_ONE_CHAIN = 4, /* the same, one chain warp takes every update
                                     (no hand-over between chain warps)                */
    SR_OT_EPOCH_SPECULATIVE_SPLIT = 5  /* the same, two preparer warps take the look-ahead
                                     of each update and one decider warp decides and
                                     applies every update                             */
} sr_ot_epoch_kernel;

typedef struct {
    int variant;              /* sr_ot_variant                                     */
    int order;                /* sr_ot_order (ignored by SR_OT_FW)                 */
    int step;                 /* sr_ot_step                                        */
    int precision;            /* sr_ot_precision                                   */
    double rho;               /* penalty weight rho = 1/lambda_paper, finite, >= 0 */
    double tol_rel_gap;       /* stop when g(T) <= tol * f(T); 0 = run max_epochs  */
    long long max_epochs;     /* epochs of m block updates (FW: iterations), >= 0 */
    int gap_every;            /* certificate every this many epochs, >= 1          */
    int refresh_every;        /* FP32: reload the running residual from the exact
                                 column sums every this many certificates; 0 never */
    int ga_M;                 /* gap-adaptive: global gap update every ga_M epochs */
    int ga_global_only;       /* gap-adaptive: 1 = no inner update (BCFW-GAS)      */
    unsigned long long seed;  /* block-order random stream                         */
    int *trace;               /* optional DEVICE int32[4*trace_capacity]: per block
                                 update k, trace[4k..4k+3] = block i, LMO vertex
                                 j*, v | dir << 29 (away vertex v in bits 0..28,
                                 all ones if none; the step's direction dir in
                                 bits 29..30: 0 toward j*, 1 away from v, 2
                                 pairwise, 3 no step), step gamma as IEEE-754
                                 binary32 bits                                    */
    long long trace_capacity;
    int dense_only;           /* 1: FP32 away/pairwise solves keep the dense row
                                 kernel instead of the active-set kernel          */
    int epoch_kernel;         /* FP32 pairwise (BCPFW) solves, one of
                                 sr_ot_epoch_kernel: which active-set kernel
                                 runs an epoch. All make the same decisions bit
                                 for bit; AUTO takes the first that applies of
                                 SPECULATIVE (d = 3 points, cyclic or permuted
                                 order, n <= 4096; or a given cost C, also the
                                 BF16 one, cyclic or permuted, n <= 8192 a
                                 multiple of 4, rows 16-byte aligned),
                                 SPECULATIVE_SPLIT (d = 3 points, uniform
                                 order, n <= 4096), PIPELINED (n <= 8192),
                                 TWO_PHASE. A kernel that does not apply falls
                                 back the same way. In sr_ot_solve_batched,
                                 TWO_PHASE selects the persistent two-phase
                                 kernel, any other value the batched
                                 speculative form (pairwise steps, cyclic or
                                 uniform order).                               */
    int cost_kind;            /* cost from points X, Y: SR_OT_COST_SQUARED
                                 (default) or SR_OT_COST_EUCLIDEAN, the paper's
                                 ||x_i - y_j||_2 (Sec. 5.1), built once into the
                                 handle's workspace (m x n) and solved as a
                                 given cost. Ignored when C is given.
                                 sr_ot_solve_batched, the point gradients dX,
                                 dY of sr_ot_grad, the BF16 cost and the points
                                 form of sr_ot_gap_noalloc take the squared
                                 cost only (EUNSUPPORTED otherwise).           */
    long long spin_limit;     /* device waits of the speculative epoch kernel
                                 (mbarrier hand-overs between its warps, and
                                 start_gate) give up after this many probes:
                                 the kernel then stops, records the timeout and
                                 the call returns SR_OT_ETIMEOUT with the handle
                                 still usable. 0 = the default, 2^26 probes
                                 (well above any legitimate wait). >= 0.       */
    int batch_warm_start;     /* sr_ot_solve_batched only: 1 = every instance
                                 starts from the feasible plan the caller left
                                 in T (rows summing to a), 0 = from T0
                                 (sr_ot_solve has its own warm_start argument) */
    const int *start_gate;    /* optional DEVICE int: the speculative epoch
                                 kernel waits (bounded by spin_limit) until it
                                 reads non-zero there before its first update;
                                 NULL = no gate. It lets the timeout path be
                                 exercised: a gate that nothing opens makes the
                                 call return SR_OT_ETIMEOUT.                   */
    int cert_schedule;        /* sr_ot_solve: 0 = a certificate (Thm 2) every
                                 gap_every epochs, as the paper evaluates it;
                                 1 = with tol_rel_gap > 0, the next certificate
                                 when the gap's geometric decay since the last
                                 one predicts the tolerance (after 1 to 8
                                 periods of gap_every epochs); the stopping
                                 decision is the exact certificate's either way.
                                 Not for SR_OT_GAP_ADAPTIVE.                   */
} sr_ot_options;

typedef struct {
    double objective;         /* f(T) at return                                    */
    double gap;               /* g(T) at return (Thm 2)                            */
    double rel_gap;           /* g / f                                             */
    double dual;              /* Lagrangian dual value w(T) = f - g (Thm 2)        */
    double row_err;           /* max_i |sum_j T_ij - a_i| / a_i; the stopping test
                                 also needs row_err <= 1e-5 (FP32 plans drift)    */
    long long epochs;         /* epochs (FW: iterations) performed                 */
    long long block_updates;  /* block updates performed                           */
    int status;               /* sr_ot_status of this solve                        */
    int reserved;
} sr_ot_result;

/* Fill *opts with defaults: BCFW, cyclic, DEC, FP32, rho = 10, tol 0,
 * max_epochs 100, gap_every 1, refresh_every 1, ga_M 1, seed 0, no trace,
 * dense_only 0, spin_limit 0 (default bound), no start gate. */
void sr_ot_default_options(sr_ot_options *opts);

/* Create a handle bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). *h is NULL on error. */
sr_ot_status sr_ot_create(sr_ot_handle *h, int device, void *cuda_stream);

/* Rebind the handle to another stream of the same device. */
sr_ot_status sr_ot_set_stream(sr_ot_handle h, void *cuda_stream);

/* Free the handle's workspace, graphs and pinned buffers. NULL is a no-op. */
sr_ot_status sr_ot_destroy(sr_ot_handle h);

/* Message for the last error on h (or for a failed sr_ot_create when h is
 * NULL). The string is owned by the library and valid until the next call. */
const char *sr_ot_last_error(sr_ot_handle h);

/*
 * Solve one instance (Alg. 1 / A.2 / A.3 / A.4 / A.1 per opts).
 *
 * Cost: exactly one of {C} (m x n) or {X (m x d), Y (n x d)} is non-NULL.
 * Points are turned into the squared-Euclidean cost C_ij = ||x_i - y_j||^2;
 * d = 3 is evaluated on the fly inside the solver, other d are materialised
 * once per call in the handle's workspace.
 * a (m), b (n): nonnegative finite weights (the paper's are histograms).
 * T_inout (m x n): if warm_start != 0, a feasible start (T >= 0, rows sum to
 * a); otherwise it is overwritten with T0 = (a_i e_0) (Thm 1). On return it
 * holds the final plan.
 * res: host pointer, filled on return.
 * Limits: block-coordinate variants take n <= 8192 (FP32) or n <= 2048
 * (FP64); SR_OT_GAP_ADAPTIVE also needs m <= 262144 (the draw walks a tree
 * of sums of the gaps held in shared memory: chunks of 32 rows, and past 8192
 * rows super nodes of 32 chunks; the per-row gaps are refreshed by a
 * certificate pass every ga_M epochs, or every epoch with ga_global_only). SR_OT_FW has no size limit beyond memory: each iteration
 * is a certificate pass (which gives every row's LMO vertex and the gap) and
 * one pass over T, so gap_every is not used.
 */
sr_ot_status sr_ot_solve(sr_ot_handle h, const sr_ot_options *opts, int m, int n, int d,
                         const void *C, const void *X, const void *Y, const void *a,
                         const void *b, void *T_inout, int warm_start, sr_ot_result *res);

/*
 * Solve `batch` independent instances in one persistent launch (captured in a
 * CUDA graph and replayed for a repeated shape set). Points mode with d = 3.
 * Pairwise steps in cyclic or uniform order run the batched speculative
 * form: one CTA solves each instance (n <= 4096; instances with more rows
 * start first) and takes its certificate when the gap's geometric decay
 * predicts the tolerance (1 to 8 periods of gap_every epochs). The other variants run a persistent two-phase kernel
 * whose instances check their certificate every gap_every epochs, or 2, 4
 * or 8 times less often while the last relative gap was more than 10, 100 or
 * 1000 times tol_rel_gap (a certificate reads the instance's whole plan).
 * m[k], n[k]: HOST arrays of per-instance sizes. off_X, off_Y, off_a, off_b,
 * off_T: HOST arrays of per-instance ELEMENT offsets into the packed device
 * buffers X, Y, a, b, T. Each instance starts from T0 = (a_i e_0), or with
 * opts->batch_warm_start from the plan in T (the tile autotuner then does not
 * run: it would write the plans).
 * res: HOST array of `batch` results; each instance has its own status.
 */
sr_ot_status sr_ot_solve_batched(sr_ot_handle h, const sr_ot_options *opts, int batch,
                                 const int *m, const int *n, int d, const long long *off_X,
                                 const long long *off_Y, const long long *off_a,
                                 const long long *off_b, const long long *off_T,
                                 const void *X, const void *Y, const void *a, const void *b,
                                 void *T, sr_ot_result *res);

/*
 * Gradients of the optimal value through the envelope theorem at a (converged)
 * plan T, for the squared-Euclidean point cost C_ij = ||x_i - y_j||^2. The
 * paper does not differentiate its solver; at an optimum the derivative of
 * the optimal value of the problem of Sec. 2 is the partial derivative of the
 * objective at fixed T:
 *   dC = T,  dX = 2 (diag(T 1) X - T Y),  dY = 2 (diag(T^T 1) Y - T^T X),
 *   db = -rho (T^T 1 - b).
 * All pointers are DEVICE pointers in opts->precision (double for SR_OT_FP64,
 * float otherwise), row-major: X (m x d), Y (n x d), b (n), T (m x n); the
 * caller owns every buffer. Any output may be NULL to skip it. X and Y are
 * needed for dX or dY (1 <= d <= 31), b for db; a is unused (kept for the
 * signature of sr_ot_solve). T is read once; partial sums are reduced in a
 * fixed order in FP64, so results are deterministic. Uses opts->precision and
 * opts->rho only. Errors: SR_OT_EINVAL (NULL/size/offset problems),
 * SR_OT_EUNSUPPORTED (d out of range), SR_OT_ENOMEM, SR_OT_ECUDA. Returns
 * after the stream has synchronised.
 */
sr_ot_status sr_ot_grad(sr_ot_handle h, const sr_ot_options *opts, int m, int n, int d,
                        const void *X, const void *Y, const void *a, const void *b,
                        const void *T, void *dC, void *dX, void *dY, void *db);

/* Batched form of sr_ot_grad over packed instances, one launch for all.
 * m, n, off_X, off_Y, off_b, off_T: HOST arrays (ELEMENT offsets, as in
 * sr_ot_solve_batched). The outputs are packed like the inputs: dX uses the
 * offsets of X, dY those of Y, db those of b. No dC output. */
sr_ot_status sr_ot_grad_batched(sr_ot_handle h, const sr_ot_options *opts, int batch,
                                const int *m, const int *n, int d, const long long *off_X,
                                const long long *off_Y, const long long *off_b,
                                const long long *off_T, const void *X, const void *Y,
                                const void *b, const void *T, void *dX, void *dY, void *db);

/* Colour-transfer tail (Sec. 5.1) and the evaluation metrics (iii), (iv) of
   Sec. 5, from one pass over a plan T (the pass of sr_ot_grad):
     Xhat_i   = sum_j T_ij y_j / sum_j T_ij      (the barycentric projection of
                source row i, the minimiser of sum_j T_ij ||x - y_j||^2; rows
                that carry no mass get zeros),
     row_err  = ||T 1 - a||_2,  col_err = ||T^T 1 - b||_2,
     e_c      = row_err + col_err,
     sparsity = the fraction of entries of T equal to zero.
   Device pointers, row-major, element type FP64 when opts->precision is
   SR_OT_FP64 and FP32 otherwise: Y (n x d, may be NULL when Xhat is NULL),
   a (m), b (n), T (m x n), Xhat (m x d, caller-owned, may be NULL). stats: a
   host struct filled when the call returns (may be NULL; a and b may then be
   NULL). Sums are taken in a fixed order (the result does not depend on
   scheduling). Errors: EINVAL for NULL T, non-positive sizes, Xhat without
   Y, stats without a or b; EUNSUPPORTED for d outside 1..31 when Xhat is
   requested. */
typedef struct {
    double e_c;       /* ||T 1 - a||_2 + ||T^T 1 - b||_2                         */
    double row_err;   /* ||T 1 - a||_2                                            */
    double col_err;   /* ||T^T 1 - b||_2                                          */
    double sparsity;  /* zero entries of T / (m n)                                */
} sr_ot_transfer_stats;

sr_ot_status sr_ot_transfer(sr_ot_handle h, const sr_ot_options *opts, int m, int n, int d,
                            const void *Y, const void *a, const void *b, const void *T,
                            void *Xhat, sr_ot_transfer_stats *stats);

/* Batched form of sr_ot_transfer over packed instances (element offsets as in
   sr_ot_solve_batched; Xhat is laid out like X: instance k's projection
   starts at off_X[k]), one pass for all. stats: host array of `batch`
   structs, or NULL. */
sr_ot_status sr_ot_transfer_batched(sr_ot_handle h, const sr_ot_options *opts, int batch,
                                    const int *m, const int *n, int d, const long long *off_X,
                                    const long long *off_Y, const long long *off_a,
                                    const long long *off_b, const long long *off_T, const void *Y,
                                    const void *a, const void *b, const void *T, void *Xhat,
                                    sr_ot_transfer_stats *stats);

/*
 * Evaluation metrics (v) and (vi) of Sec. 5: the distance of a plan T from a
 * reference plan T_lp, which the paper takes as T*_LP, the optimal plan of
 * the unrelaxed transport problem (min <C, T> over T >= 0, T 1 = a,
 * T^T 1 = b; the caller computes it with any exact OT solver):
 *   e_m = ||T - T_lp||_F / ||T_lp||_F,
 *   e_v = |<T, C> - <T_lp, C>| / |<T_lp, C>|.
 * Cost as in sr_ot_gap: exactly one of C (m x n) or d = 3 points X, Y (the
 * squared cost, or the Euclidean one with SR_OT_COST_EUCLIDEAN, evaluated on
 * the fly as the solver evaluates it); other d: pass C (SR_OT_EUNSUPPORTED).
 * DEVICE pointers, row-major, FP64 for SR_OT_FP64 and FP32 otherwise. One
 * pass over T and T_lp; FP32 products are summed with compensation per lane
 * and in FP64 across lanes, in a fixed order (deterministic). Uses
 * opts->precision and opts->cost_kind only. out: HOST struct, filled when the
 * call returns. Errors: EINVAL (NULL pointers, sizes, both or neither cost
 * source), EUNSUPPORTED (points with d != 3), ENOMEM, ECUDA.
 */
typedef struct {
    double e_m;        /* ||T - T_lp||_F / ||T_lp||_F                        */
    double e_v;        /* |<T, C> - <T_lp, C>| / |<T_lp, C>|                 */
    double diff_norm;  /* ||T - T_lp||_F                                     */
    double lp_norm;    /* ||T_lp||_F                                         */
    double value;      /* <T, C>                                             */
    double lp_value;   /* <T_lp, C>                                          */
} sr_ot_lp_metrics_result;

sr_ot_status sr_ot_lp_metrics(sr_ot_handle h, const sr_ot_options *opts, int m, int n, int d,
                              const void *C, const void *X, const void *Y, const void *T,
                              const void *T_lp, sr_ot_lp_metrics_result *out);

/*
 * Certificate of any feasible plan T (Thm 2): objective f, linearisation
 * duality gap g = sum_i g_i (eq. 11) and Lagrangian dual w = f - g.
 * Cost as in sr_ot_solve. If g_rows is non-NULL it receives the per-row
 * gaps g_i as DEVICE doubles (m). Uses opts->precision and opts->rho only.
 */
sr_ot_status sr_ot_gap(sr_ot_handle h, const sr_ot_options *opts, int m, int n, int d,
                       const void *C, const void *X, const void *Y, const void *a,
                       const void *b, const void *T, double *g_rows, sr_ot_result *res);

/*
 * Squared-Euclidean cost matrix C_ij = ||x_i - y_j||^2 (m x n, float),
 * built on the tensor cores from BF16-rounded points with FP32 accumulation
 * and FP32 norms of the rounded points: C = |x~|^2 + |y~|^2 - 2 X~ Y~^T.
 * X (m x d), Y (n x d) are float; d must be a multiple of 64. The paper uses
 * the Euclidean cost of colour centroids (Sec. 5.1); the GEMM form is this
 * library's route for feature dimensions d >= 64.
 */
sr_ot_status sr_ot_cost_bf16(sr_ot_handle h, int m, int n, int d, const float *X,
                             const float *Y, float *C);

/*
 * The certificate of sr_ot_gap for callers that cannot allocate device
 * memory where they need it: an application whose caching allocator has
 * reserved the device's memory up front, a plug-in inside a host program
 * that owns every allocation, a long-running service that must not fail on
 * fragmentation after start-up. The paper has no counterpart; this is an
 * interface of this library only.
 *
 * It takes no handle and allocates nothing: no cudaMalloc/cudaFree, no
 * pinned buffer. Its scratch is a fixed 4 MiB array compiled into the
 * library as a static __device__ variable, present on every device that
 * loads the library until the process exits. Every n <= 207,552 fits for
 * any m (smaller m leave room for slightly larger n); sizes that do not fit
 * fail with SR_OT_EUNSUPPORTED and a message naming the bytes needed. The
 * cost must be C or d = 3 points (squared cost only: with
 * SR_OT_COST_EUCLIDEAN pass the cost as C, else SR_OT_EUNSUPPORTED);
 * precision SR_OT_FP64 or SR_OT_FP32.
 *
 * `device` must be the device the pointers live on; `cuda_stream` as in
 * sr_ot_create. The calling thread's current device is the same before and
 * after the call. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture. The call synchronises `cuda_stream` before it returns (it reads
 * the input checks and the certificate back to the host). Every call
 * reuses the same array and leaves its last contents there, so calls whose
 * kernels overlap on the GPU race: serialise them. Arguments, outputs (res
 * on the host, g_rows optional device doubles) and errors are as for
 * sr_ot_gap; the error message is sr_ot_last_error(NULL).
 */
sr_ot_status sr_ot_gap_noalloc(int device, void *cuda_stream, const sr_ot_options *opts, int m,
                               int n, int d, const void *C, const void *X, const void *Y,
                               const void *a, const void *b, const void *T, double *g_rows,
                               sr_ot_result *res);

/*
 * Observability (not in the paper). sr_ot_launch_count: number of this
 * library's kernels launched on h since it was created. When profiling is
 * enabled, the library brackets each launch group on the handle's stream with
 * CUDA events and accumulates device time per kernel class:
 *   SR_OT_PROF_EPOCH  single-instance epoch kernels (block updates)
 *   SR_OT_PROF_CERT   certificate passes (column sums, row pass, reduction)
 *   SR_OT_PROF_BATCH  batched persistent solves
 *   SR_OT_PROF_GRAD   adjoint kernels
 *   SR_OT_PROF_COST   cost materialisation (plain or BF16 tensor-core GEMM)
 *   SR_OT_PROF_METRICS  the pass of sr_ot_lp_metrics
 * sr_ot_profile_read returns the total milliseconds and the number of timed
 * launch groups of one class; sr_ot_profile_enable(h, 1) also resets them.
 */
enum { SR_OT_PROF_EPOCH = 0, SR_OT_PROF_CERT = 1, SR_OT_PROF_BATCH = 2, SR_OT_PROF_GRAD = 3,
       SR_OT_PROF_COST = 4, SR_OT_PROF_METRICS = 5, SR_OT_PROF_KINDS = 6 };
long long sr_ot_launch_count(sr_ot_handle h);

/*
 * Latency floor of the speculative epoch kernel's update chain (observability,
 * not in the paper). One CTA runs `updates` (>= 1) dependent updates that keep
 * only what the solver's chain keeps: read the residual at the two columns the
 * previous update changed, compare-select, form the pairwise step, write the
 * residual of two columns, publish; with `chain_warps` = 3 the updates rotate
 * over three warps that hand over through mbarriers as the solver's do, with
 * 1 one warp runs them all. *ns_per_update receives the device time per update
 * (CUDA events on the handle's stream around the launch). Errors: EINVAL
 * (chain_warps not 1 or 3, updates < 1, NULL output), ETIMEOUT, ECUDA.
 */
sr_ot_status sr_ot_profile_chain_floor(sr_ot_handle h, int chain_warps, int updates, double *ns_per_update);
sr_ot_status sr_ot_profile_enable(sr_ot_handle h, int enable);
sr_ot_status sr_ot_profile_read(sr_ot_handle h, int kind, double *total_ms, long long *groups);

#ifdef __cplusplus
}
#endif
#endif /* SR_OT_H */
