/*
 * gmco.h - C ABI of the batched gL-BFGS Pareto-plan optimiser for HDR prostate
 * brachytherapy on NVIDIA B300 (sm_103a).
 *
 * Method: Belanger, Cui et al., "A GPU-based multi-criteria optimization algorithm for HDR
 * brachytherapy" (arXiv 1904.01567).  Each plan p of a batch has its own hidden weights w_p
 * (Eq. (obj)); the library minimises, for every plan at once,
 *
 *     F_p(x) = sum_s w_ps / N_s  sum_{i in s} f_s(d_i),      d = A t,   t = x*x,
 *
 * with f_s the piecewise quadratic penalty of Eq. (1), the dose of Eq. (dose), the
 * non-negativity substitution t = x^2 of Sec. 2.1.2 and the gradient of Eq. (2), by
 * limited-memory BFGS (Sec. 2.2.2) with a backtracking Armijo line search, stopping on the
 * relative variation of the objective (Sec. 2.2.3).  DVH indices follow Sec. 2.3.1.
 *
 * Conventions for every call:
 *   - Pointers may be host or device memory (checked with cudaPointerGetAttributes).
 *     Host buffers are staged through device memory inside the call.
 *   - All matrices are row-major.  Batched per-plan data is plan-major: row p holds plan p
 *     (so T, an n_dwell x P matrix with one column per plan, is stored as P x n_dwell).
 *   - Calls return a gmco_status and never abort or throw; per-plan numerical outcomes are
 *     reported as gmco_plan_status values.
 *   - One problem is used by one host thread and one stream at a time.  Calls that take a
 *     stream run on it and return after their results are in the caller's buffers.
 *   - Nothing falls back to the CPU: without a usable CUDA device every call that needs one
 *     returns GMCO_ECUDA.
 */
#ifndef GMCO_H
#define GMCO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gmco_problem gmco_problem;
typedef struct gmco_multi gmco_multi;

typedef enum {
    GMCO_OK = 0,
    GMCO_EINVAL = 1,       /* bad shape, null pointer, non-finite or negative input */
    GMCO_ENOMEM = 2,       /* device allocation failed */
    GMCO_ECUDA = 3,        /* CUDA runtime error, or no usable device */
    GMCO_ETIMEOUT = 4,     /* the solve hit its step budget with plans still running */
    GMCO_EUNSUPPORTED = 5  /* valid request this build cannot serve (e.g. too many dwells) */
} gmco_status;

typedef enum {
    GMCO_PLAN_CONVERGED = 0, /* relative objective change <= tol, F == 0 or gradient == 0 */
    GMCO_PLAN_MAXITER = 1,   /* max_iters accepted iterations without meeting tol */
    GMCO_PLAN_LSFAIL = 2,    /* line search failed along steepest descent; x kept */
    GMCO_PLAN_NONFINITE = 3  /* objective or gradient not finite */
} gmco_plan_status;

typedef enum {
    GMCO_PREC_FP32 = 0,   /* A in FP32, FP32 SIMT dose and gradient contractions */
    GMCO_PREC_BF16 = 1,   /* A in BF16 with a per-point power-of-two scale; tcgen05 BF16 MMA
                             (FP32 accumulate) with two-term BF16 splits of t and of dF/dd */
    GMCO_PREC_FP8 = 2,    /* A quantised to FP8 E4M3 with a per-point power-of-two scale, run
                             on the BF16 tensor-core path (E4M3 values are exact in BF16) */
    GMCO_PREC_BF16X2 = 3, /* A, t and dF/dd each split into two BF16 terms (about 16 bits) */
    GMCO_PREC_BF16X3 = 4  /* three BF16 terms each (24 bits, the FP32 significand): products
                             with term orders i + j <= 4, FP32 accuracy on the tensor cores */
} gmco_precision;

/* Number of DVH indices written per plan, in this order (Sec. 2.3.1; structure 0 is the
 * target, 1 the urethra, 2 and 3 the rectum and bladder):
 *   0 V100 of structure 0, % of its points receiving >= rx_gy
 *   1 D90  of structure 0, % of rx_gy (k-th largest dose, k = ceil(0.9 N_0))
 *   2 D10  of structure 1, % of rx_gy (k = ceil(0.1 N_1))
 *   3 V75  of structure 2, % of its points receiving >= 0.75 rx_gy
 *   4 V75  of structure 3, same
 * Indices of absent structures are NaN. */
#define GMCO_DVH_K 5

typedef struct {
    int32_t precision;     /* gmco_precision, default GMCO_PREC_FP32 */
    int32_t m;             /* L-BFGS history pairs, 1..16, default 10 */
    double c1;             /* Armijo sufficient-decrease constant, default 1e-4 */
    int32_t max_ls;        /* line-search trials per direction, 1..60, default 30 */
    double rx_gy;          /* prescription dose for the DVH indices, default 15 Gy */
    int32_t refine_iters;  /* after a BF16/FP8 solve, up to this many further iterations
                              with the FP32 evaluation (history kept); default 0 */
    int32_t steps_per_poll;/* device steps between host checks for completion, default 16 */
    int32_t stop_window;   /* a plan converges after this many consecutive accepted
                              iterations each with |F_prev - F| <= tol |F_prev|; default 1 */
    int32_t grad_split_kb; /* tensor-core forms: points per split of the gradient GEMM, in
                              blocks of 64 points (each split's partial sums are added in a
                              fixed order); 0 (default) = chosen from the row count so that
                              about one wave of splits covers the GPU */
    int32_t max_evals;     /* objective evaluations per plan (the first one and every
                              line-search trial), >= 0; a plan that would exceed it stops at
                              its last accepted point with GMCO_PLAN_MAXITER.  Every batched
                              step evaluates each running plan once, so this bounds the
                              steps of a solve.  0 (default) = no limit */
    int32_t grad_plan_tile;/* tensor-core forms: plans per gradient-GEMM tile, 128 or 256 (one
                              MMA of N = 256 per product where a stage of 256 fits), or 0
                              (default) for 256 where it fits, else 128 */
    int32_t sparse_grad_permille; /* tensor-core forms, solver steps of a single problem: a
                              step whose previous step had at most this many active (plan,
                              point) pairs per thousand (penalty term on, dF/dd != 0) forms
                              the gradient from the active pairs alone, in FP32, instead of
                              the gradient GEMM.  0..1000; 0 (default) = always the GEMM.
                              At about 1% active pairs the two cost about the same: each
                              active pair reads a whole row of A, where the GEMM reuses it */
    int32_t wait_limit_us; /* tensor-core forms: every wait inside the GEMM kernels (a stage of
                              operands landing, an accumulator handed between the MMA issuer
                              and the epilogue) gives up after this many microseconds; the
                              kernel then waits (at most 1 s more) for its own copies and MMAs
                              in flight, frees its tensor memory and exits, and the call
                              returns GMCO_ECUDA.  1..60000000; default 1000000 (1 s).  No
                              wait takes longer than a few microseconds in a correct run, so
                              only a fault elsewhere (or a limit set far too short, as a test
                              does) ever reaches it */
} gmco_options;

/* Fills *opt with the defaults above. */
void gmco_default_options(gmco_options *opt);

/* ---- dose rate matrix ----
 * Step (i) of the GPU planning flow (Sec. 2.2.1): the dose rate of every dwell position at
 * every dose calculation point, the A of Eq. (dose).  The paper does not state its dose-rate
 * model; this is the isotropic point source
 *   A_il = lambda * sk * unit * g(r) / r^2,  r = max(|p_i - q_l|, r_min),  g = g0 + g1 r + g2 r^2,
 * with r in cm.  Defaults (gmco_default_source): lambda = 1.109 cGy h^-1 U^-1, sk = 40700 U,
 * unit = 1 / 360000 (cGy/h to Gy/s, so that dwell times are seconds), r_min = 0.1 cm,
 * g = 1 + 0.005 r - 0.002 r^2. */
typedef struct gmco_source {
    double lambda, sk, unit, r_min, g0, g1, g2;
} gmco_source;

void gmco_default_source(gmco_source *src);

/* Computes A on the current device in FP32.
 *   points   n_pnt x 3 dose calculation point coordinates, cm (host or device, row-major)
 *   dwells   n_dwell x 3 dwell position coordinates, cm (host or device)
 *   src      the model, or NULL for the defaults
 *   A_out    n_pnt x n_dwell, row-major, Gy/s (host or device; the layout gmco_create_problem
 *            takes, which accepts the device buffer directly)
 * 1 <= n_dwell <= 1024, 1 <= n_pnt <= 2^31.  Returns GMCO_EINVAL for bad sizes, NULL pointers,
 * non-finite model constants or coordinates, r_min <= 0, or a distance where g(r) <= 0 (the
 * model's radial fit is negative beyond about 23.6 cm).  Queued on cuda_stream (NULL: the
 * default stream) and complete on return. */
gmco_status gmco_dose_rate_matrix(const float *points, int64_t n_pnt, const float *dwells,
                                  int64_t n_dwell, const gmco_source *src, float *A_out,
                                  void *cuda_stream);

/* Dose calculation points of the workload's analytic structures (the sampling half of step
 * (i); the clinical flow creates points from contours, which needs DICOM data): structure 0
 * the prostate ellipsoid (semi-axes a, b, c at the origin) without the urethra, 1 the urethra
 * (cylinder of radius urethra_r on the z axis, |z| <= c), 2 the rectum (cylinder of radius
 * rectum_r parallel to z through (0, rectum_y), |z| <= rectum_half_len) outside the prostate,
 * 3 the bladder (sphere of radius bladder_r at (0, 0, bladder_z)) outside the prostate and
 * the rectum.  Sizes in cm.
 * Rule (uniform rejection sampling with a counter-based generator, reproducible anywhere):
 * candidate k of structure s is lo + u w in the structure's bounding box (corner lo, widths w,
 * per axis), u = top 24 bits of SplitMix64 output s 2^40 + 4 k + axis (axis 0, 1, 2 = x, y, z)
 * seeded with `seed`, times 2^-24; point i of structure s is its i-th accepted candidate.  The
 * geometry is rounded to FP32 and every arithmetic step is one IEEE FP32 operation in a fixed
 * order (see points.cu), so the points are reproducible bit for bit.
 *   counts   4 point counts (>= 0, total 1..2^31)
 *   points   sum(counts) x 3 FP32 coordinates, structure-major (host or device)
 *   sid      sum(counts) structure ids 0..3 (host or device)
 * GMCO_EINVAL for non-finite or non-positive sizes, bad counts, NULL pointers, or a structure
 * that accepts too few candidates (empty, or covered by what it excludes).  Synchronous on
 * cuda_stream. */
typedef struct gmco_geometry {
    double a, b, c;                              /* prostate semi-axes */
    double urethra_r;
    double rectum_r, rectum_y, rectum_half_len;
    double bladder_r, bladder_z;
} gmco_geometry;

gmco_status gmco_sample_points(const gmco_geometry *geo, const int64_t *counts, uint64_t seed,
                               float *points, int32_t *sid, void *cuda_stream);

/* Creates a problem on the current CUDA device.
 *   A               n_pnt x n_dwell dose-rate matrix, Gy/s, finite and >= 0 (Eq. (dose));
 *                   copied (and quantised for BF16/FP8), the caller may free it afterwards
 *   structure_ids   n_pnt values in [0, n_struct); every structure needs >= 1 point
 *   penalty_params  n_struct x 4: (w_min, D_min, D_max, w_max) of Eq. (1), Gy; weights
 *                   finite and >= 0, D_min <= D_max, D_min may be -inf, D_max may be +inf
 *   opt             options, or NULL for the defaults
 * 1 <= n_dwell <= 1024, 1 <= n_pnt, 1 <= n_struct <= 16; the tensor-core precisions need
 * n_dwell <= 512 and n_struct <= 8 (GMCO_EUNSUPPORTED otherwise).  Returns GMCO_EINVAL on bad
 * arguments, GMCO_ENOMEM / GMCO_ECUDA on device failure; *out is NULL unless GMCO_OK. */
gmco_status gmco_create_problem(const float *A, int64_t n_pnt, int64_t n_dwell,
                                const int32_t *structure_ids, int32_t n_struct,
                                const double *penalty_params, const gmco_options *opt,
                                gmco_problem **out);

/* Releases every device buffer of the problem.  NULL is allowed. */
void gmco_destroy_problem(gmco_problem *prob);

/* Solves P plans at once (gMCO, Sec. 2.3.2): plan p minimises F_p with hidden weights
 * penalty_weights[p, :] from the start t0[p, :].
 *   penalty_weights P x n_struct, finite and >= 0
 *   t0              P x n_dwell start dwell times (s), finite and >= 0, or NULL for 1 s
 *   max_iters       accepted iterations per plan, >= 0
 *   tol             relative objective change that ends a plan, >= 0
 * Outputs (any may be NULL except none of them needs to be given):
 *   T_out           P x n_dwell final dwell times t = x^2 (s)
 *   objectives      P final objectives F_p; with BF16/FP8 precision they are re-evaluated
 *                   with the FP32 path at the final T
 *   dvh             P x GMCO_DVH_K indices of the final doses (FP32 path)
 *   iters_out       P accepted iterations
 *   plan_status     P gmco_plan_status values
 * Returns GMCO_ETIMEOUT when plans were still running after the step budget
 * (max_iters * (max_ls + 1) + 2 steps); outputs then hold the current iterates. */
gmco_status gmco_solve_batch(gmco_problem *prob, const float *penalty_weights, int64_t P,
                             const float *t0, int32_t max_iters, double tol, float *T_out,
                             double *objectives, float *dvh, int32_t *iters_out,
                             int32_t *plan_status, void *cuda_stream);

/* One evaluation at given dwell weights X (P x n_dwell), with the problem's precision:
 *   objectives  P values of Eq. (obj)
 *   grad_x      P x n_dwell gradient of Eq. (2) summed over points (dF/dx)
 *   dose        P x n_pnt doses of Eq. (dose)
 *   dvh         P x GMCO_DVH_K DVH indices of those doses
 * Any output may be NULL.  All outputs come from the problem's precision form (the dose of
 * a tensor-core form is that form's dose GEMM), so this call measures each form's error. */
gmco_status gmco_evaluate(gmco_problem *prob, const float *penalty_weights, int64_t P,
                          const float *X, double *objectives, float *grad_x, float *dose,
                          float *dvh, void *cuda_stream);

/* The stochastic engine gSA (Sec. 2.2.1, steps (ii)-(v) repeated), the paper's second GPU
 * engine, for comparison with gmco_solve_batch.  The paper gives neither its move nor its
 * cooling schedule; this engine's, with f = k / (iterations - 1) over iterations k:
 *   start x = sqrt(t0) (t0 NULL: 1 s);
 *   move   x'_l = x_l + delta_k (2 u - 1) for every dwell l of every plan, t = x'^2,
 *          delta_k = step0 (step_final / step0)^f;
 *   accept when F(x') - F(x) <= -T_k F(x_0) ln v, T_k = T0 (T_final / T0)^f (temperatures are
 *          fractions of the plan's start objective);
 * u and v are uniform draws: the top 53 bits of output n of SplitMix64 (Steele, Lea and Flood
 * 2014) seeded with `seed`, times 2^-53 (u in [0, 1)), plus one (v in (0, 1]), at
 * n = k 2^42 + p 2^21 + l for plan p (its row in this call) and dwell l (l = 2^21 - 1: v).
 * Every objective is the problem's precision form (the same kernels as gmco_evaluate).
 *   iterations  0 <= K < 2^22; seed any value; T0, T_final, step0, step_final finite and
 *               >= 0, with T0 = 0 exactly when T_final = 0 (and the same for the steps)
 * Outputs (any may be NULL): T_out (P x n_dwell) the best dwell times seen, objectives (P) their
 * objectives, accepts (P) the accepted moves.  n_dwell < 2^21 - 1 and P < 2^21. */
typedef struct {
    int32_t iterations;      /* default 1000 */
    uint64_t seed;           /* default 1 */
    double T0, T_final;      /* default 1e-2, 1e-5 */
    double step0, step_final;/* default 0.2, 0.002 (units of x = sqrt(t), sqrt(s)) */
} gmco_sa_options;

void gmco_default_sa_options(gmco_sa_options *opt);

gmco_status gmco_solve_sa(gmco_problem *prob, const float *penalty_weights, int64_t P,
                          const float *t0, const gmco_sa_options *opt, float *T_out,
                          double *objectives, int32_t *accepts, void *cuda_stream);

/* Allocation-free variant of gmco_evaluate, for callers that cannot allocate device memory
 * while they run (a fixed memory budget, a real-time loop that cannot take cudaMalloc's
 * implicit synchronisation, an application that owns every allocation).  The paper has no
 * counterpart; it is an interface addition.
 *   Computes objectives[P] and grad_x[P x n_dwell] (either may be NULL, not both) at dwell
 *   weights X[P x n_dwell] with weights penalty_weights[P x n_struct], always with the FP32
 *   form (the problem's FP32 copy of A), whatever the problem's precision.
 *   Every pointer must be device memory (GMCO_EINVAL otherwise).
 *   Scratch is one fixed 8 MiB device array inside the library, present on every GPU that
 *   loads it until the process exits; a request that needs more (about
 *   P x (n_pnt + 6 n_dwell) x 4 bytes) returns GMCO_EUNSUPPORTED and launches nothing.
 *   The first call on a device resolves that array's address on the device (once, with the
 *   device current); make that first call before any stream capture.
 *   Asynchronous: kernels are queued on cuda_stream and the call returns without waiting.
 *   All calls share the one array: calls whose kernels overlap on the GPU (different streams,
 *   or threads without ordering) race and corrupt each other.  Each call writes every scratch
 *   value before reading it, so nothing has to be cleared between calls.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library routine. */
gmco_status gmco_evaluate_noalloc(const gmco_problem *prob, const float *penalty_weights,
                                  int64_t P, const float *X, double *objectives, float *grad_x,
                                  void *cuda_stream);

/* DVH indices (GMCO_DVH_K per plan, see above) of given dwell times: T is P x n_dwell (s,
 * finite and >= 0; host or device).  The doses A t of Eq. (dose) are formed with the FP32 form
 * whatever the problem's precision, and the indices are counted exactly on them.  A problem
 * built on a separate, denser point set of the same structures and dwell positions gives the
 * DVH of plans optimised on a coarser one (Sec. 2.1: the paper evaluates DVHs on their own
 * point set).  GMCO_EINVAL for bad sizes, NULL pointers or negative / non-finite times. */
gmco_status gmco_dvh_at(gmco_problem *prob, const float *T, int64_t P, float *dvh,
                        void *cuda_stream);

/* DVH indices (GMCO_DVH_K per plan, see above) of given doses: dose is P x n_pnt (Gy).
 * Exact on the given FP32 values: counts and k-th largest values, no interpolation. */
gmco_status gmco_dvh_from_dose(gmco_problem *prob, const float *dose, int64_t P, float *dvh,
                               void *cuda_stream);

/* Measurement aid: times one evaluation of P plans at a line-search trial point
 * (x_trial = 1.01 X, so both the dose and the dose change are computed) `reps` times after
 * one warm-up, back to back on the problem's stream (as the solve loop launches them), with
 * CUDA events between its kernels.  reps is at most 1000.
 *   ms     4 averages (milliseconds): trial-point preparation, dose GEMM with the penalty
 *          epilogue, gradient GEMM, reduction of partial sums
 *   flops  4 values or NULL: algorithmic FLOPs of the dose GEMM (the dose d = A t of
 *          Eq. (dose), 2 P n_pnt n_dwell; the dose change dd it also forms for the line search
 *          is not counted) and of the gradient GEMM (2 P n_pnt n_dwell), then the FLOPs the
 *          kernels issue (tensor-core split terms of d and dd over padded tiles; for FP32 the
 *          dose kernel's d and dd, 4 P n_pnt n_dwell, and the gradient's 2 P n_pnt n_dwell).
 * Synchronous. */
gmco_status gmco_profile_evaluate(gmco_problem *prob, const float *penalty_weights, int64_t P,
                                  const float *X, int32_t reps, double *ms, double *flops);

/* Measurement aid: the device's FP32 fused multiply-add throughput in TFLOP/s, the pipe peak
 * against which the FP32 form's SIMT contractions are reported: tflops[0] with scalar FFMA
 * (the instruction the FP32 form's kernels issue), tflops[1] with paired FP32 FMA (two FP32
 * lanes per instruction).  Each is the best of `reps` launches of `iters` iterations of 16
 * independent FMA chains per thread on 8 resident blocks of 256 threads per SM, timed with CUDA
 * events.  Synchronous; uses the current device and stream 0; allocates one small buffer. */
gmco_status gmco_fp32_peak(int32_t iters, int32_t reps, double *tflops);

/* ---- plan pool post-processing ----
 * RTOG evaluation (Sec. 2.3.1: target V100 >= 90 %, urethra D10 < 118 % of the prescription,
 * bladder and rectum V75 < 1 cc; RTOG+ asks V100 >= 95 %) and the selection of one plan from
 * the pool (Sec. 2.4: RTOG+ valid first, then RTOG valid, each by the highest target V100; else
 * an invalid plan, preferring those that meet the target and urethra criteria, by the lowest
 * rectum plus bladder V75; ties go to the lower index).  The V75 of a DVH row are % of the
 * structure's points; vol_cc turns them into cc. */
typedef struct gmco_rtog {
    double v100_min;        /* % of the target, RTOG: 90 */
    double v100_min_plus;   /* RTOG+: 95 */
    double d10_max;         /* urethra D10 below this, % of the prescription: 118 */
    double v75_max_cc;      /* rectum and bladder V75 below this, cc: 1 */
    double vol_cc[2];       /* volumes of structures 2 (rectum) and 3 (bladder), cc; no default */
} gmco_rtog;

/* The protocol's values above; vol_cc set to 0 (the caller supplies the volumes). */
void gmco_default_rtog(gmco_rtog *crit);

/* dvh: P x GMCO_DVH_K rows as gmco_solve_batch writes them (host or device).  cls (P values,
 * may be NULL): 2 = RTOG+ valid, 1 = RTOG valid, 0 = invalid; *selected: index of the selected
 * plan.  Outputs host or device.  GMCO_EINVAL for P < 1, NULL dvh / selected / crit, or
 * non-finite or negative volumes.  Complete on return. */
gmco_status gmco_rtog_select(const float *dvh, int64_t P, const gmco_rtog *crit, int32_t *cls,
                             int32_t *selected, void *cuda_stream);

/* Non-dominated filter of a plan pool (Sec. 2.2.4): obj is P x K objective values (K <= 16,
 * all minimised, FP64, host or device); nondominated[i] = 1 when no plan is no worse in every
 * objective and better in one, else 0 (host or device).  Equal rows do not dominate each
 * other.  GMCO_EINVAL for bad sizes or NULL pointers.  Complete on return. */
gmco_status gmco_pareto_filter(const double *obj, int64_t P, int32_t K, int32_t *nondominated,
                               void *cuda_stream);

/* ---- several patients in one launch (uneven batching) ----
 * A gmco_multi groups 1..64 problems (patients with their own dwell and point counts) that
 * share one tensor-core precision and the same m, c1, max_ls, stop_window and
 * steps_per_poll options, on one device.  gmco_solve_multi solves every patient's batch of
 * plans together: each solver step is one dose-GEMM launch, one gradient-GEMM launch and one
 * update launch for all patients (persistent kernels that walk one list of work items:
 * patient x plan tile x point tile, and patient x plan tile x point split), captured in CUDA
 * graphs of steps_per_poll steps.  The paper solves one patient at a time; this is an
 * extension of its batched solve (Sec. 2.3.2) to many patients.
 * Results of patient p are bit for bit those of gmco_solve_batch on its own problem created
 * with options.grad_split_kb equal to the multi object's split setting (and the active-set
 * gradient off, the default: the multi launch always forms the gradient with the GEMM).
 * The multi object keeps stacked copies of the problems' BF16 terms of A; the problems must
 * outlive it and must not be used by another call while a multi call runs. */

/* probs: n problem handles (host array).  GMCO_EINVAL for mixed precisions or options, an
 * FP32-form problem (GMCO_EUNSUPPORTED), n outside 1..64 or problems on different devices. */
gmco_status gmco_create_multi(gmco_problem *const *probs, int32_t n, gmco_multi **out);

/* Releases the multi object (not its problems).  NULL is allowed. */
void gmco_destroy_multi(gmco_multi *multi);

/* Points per split of every patient's gradient GEMM, in blocks of 64 points (>= 1), or 0 for
 * each problem's own automatic choice.  The default is set by gmco_multi_autotune, else 16. */
gmco_status gmco_multi_set_split(gmco_multi *multi, int32_t split_kb);
int32_t gmco_multi_get_split(const gmco_multi *multi);

/* The launch's tiles: split length as above and plans per gradient-GEMM tile (0, 128 or 256 as
 * gmco_options.grad_plan_tile; the problems' option is the initial value).  get returns the
 * requested tile (0 = the default). */
gmco_status gmco_multi_set_tiles(gmco_multi *multi, int32_t split_kb, int32_t grad_plan_tile);
int32_t gmco_multi_get_grad_tile(const gmco_multi *multi);

/* Solves every patient's plans.  All arrays have n entries (host arrays of pointers); entry p
 * has the meaning and size of the same argument of gmco_solve_batch for patient p with P[p]
 * plans (P[p] >= 1).  t0 may be NULL (uniform start for everyone) and so may any output
 * array or any of its entries.  GMCO_ETIMEOUT as for gmco_solve_batch, when any patient hit
 * the step budget. */
gmco_status gmco_solve_multi(gmco_multi *multi, const float *const *penalty_weights,
                             const int64_t *P, const float *const *t0, int32_t max_iters,
                             double tol, float *const *T_out, double *const *objectives,
                             float *const *dvh, int32_t *const *iters_out,
                             int32_t *const *plan_status, void *cuda_stream);

/* Autotuner of the multi-patient launch: for each candidate split length (as for
 * gmco_multi_set_split) runs `steps` solver steps from the uniform start on the given
 * weights, times them with CUDA events, writes the mean milliseconds per step to
 * ms_per_step[i], selects the fastest and returns it in *best.  Synchronous. */
gmco_status gmco_multi_autotune(gmco_multi *multi, const float *const *penalty_weights,
                                const int64_t *P, int32_t steps, const int32_t *candidates,
                                int32_t n_candidates, double *ms_per_step, int32_t *best);

/* The same over tile configurations: candidate i is (split_kb[i], grad_plan_tile[i]) as for
 * gmco_multi_set_tiles.  Selects the fastest and returns its index in *best_index. */
gmco_status gmco_multi_autotune_tiles(gmco_multi *multi, const float *const *penalty_weights,
                                      const int64_t *P, int32_t steps, const int32_t *split_kb,
                                      const int32_t *grad_plan_tile, int32_t n_candidates,
                                      double *ms_per_step, int32_t *best_index);

/* Kernel launches made by the most recent gmco_solve_multi call. */
int64_t gmco_multi_last_launch_count(const gmco_multi *multi);

/* ---- learned warm start ----
 * A per-dwell-position multilayer perceptron predicts each plan's dwell times from 10
 * geometric features of the dwell position and the plan's 4 penalty weights; the solver then
 * starts from the prediction.  The paper has no learned part (it starts from uniform times,
 * Sec. 2.3.2); this is an extension.  Network:
 *     x0  = [f_1 .. f_10, log10 max(w_1, 1e-3) .. log10 max(w_4, 1e-3)]        (14 inputs)
 *     h_l = GELU(h_{l-1} W_l + b_l), l = 1..3, width 128, GELU(z) = z (1 + erf(z / sqrt 2)) / 2
 *     t   = softplus(h_3 . w_4 + b_4)      (seconds)
 * Parameters are one FP32 array of GMCO_MLP_NPARAM values in this order, matrices
 * row-major with the input index first: W_1 [14][128], b_1 [128], W_2 [128][128], b_2,
 * W_3 [128][128], b_3, w_4 [128], b_4 [1].  Products use BF16 weights and activations with
 * FP32 accumulation; FP32 master weights are updated by Adam (beta 0.9, 0.999, eps 1e-8).
 * Loss: mean over the batch rows of (t - t_target)^2.  The 10 features are the caller's
 * (computed from its contours); the library treats them as numbers. */
#define GMCO_MLP_NPARAM 35073
typedef struct gmco_mlp gmco_mlp;

/* Creates a network from initial parameters (host or device; finite). */
gmco_status gmco_mlp_create(const float *params, gmco_mlp **out);
void gmco_mlp_destroy(gmco_mlp *mlp);
/* Current FP32 master parameters. */
gmco_status gmco_mlp_get_params(gmco_mlp *mlp, float *params);

/* Checkpoint of a network and its training state, so that training resumes exactly: the file
 * holds the line "GMCO-MLP", one line of JSON (format, version 1, GMCO_MLP_NPARAM, the Adam step
 * count, the arrays, the parameter layout), then three arrays of GMCO_MLP_NPARAM little-endian
 * FP32 values: the master parameters and Adam's first and second moments.  Training steps after
 * gmco_mlp_load give the same parameters, bit for bit, as the same steps of the network that
 * was saved.  save: GMCO_EINVAL when the file cannot be written.  load: creates a network on the
 * current device; GMCO_EINVAL for a file that is missing, of another format, version or size,
 * or holds non-finite values or negative second moments (checked before any device use). */
gmco_status gmco_mlp_save(gmco_mlp *mlp, const char *path);
gmco_status gmco_mlp_load(const char *path, gmco_mlp **out);

/* Predicted dwell times of P plans of one patient: t_out[p][l] for features[l] (n_dwell x
 * 10) and penalty_weights[p] (P x 4), each at least t_floor. */
gmco_status gmco_mlp_predict(gmco_mlp *mlp, const float *features, int64_t n_dwell,
                             const float *penalty_weights, int64_t P, float t_floor,
                             float *t_out, void *cuda_stream);

/* Loss and gradient (GMCO_MLP_NPARAM values, the parameter layout) at the current weights
 * over R training rows: row r has features[pairs[r][0]] (n_feat x 10 table), penalty
 * weights penalty_weights[pairs[r][1]] (n_w x 4 table) and target dwell time target[r]. */
gmco_status gmco_mlp_gradient(gmco_mlp *mlp, const float *features, int64_t n_feat,
                              const float *penalty_weights, int64_t n_w, const int32_t *pairs,
                              const float *target, int64_t R, float *loss, float *grad,
                              void *cuda_stream);

/* One Adam step with learning rate lr on the gradient of those rows; *loss (may be NULL) is
 * the loss before the step. */
gmco_status gmco_mlp_train_step(gmco_mlp *mlp, const float *features, int64_t n_feat,
                                const float *penalty_weights, int64_t n_w, const int32_t *pairs,
                                const float *target, int64_t R, float lr, float *loss,
                                void *cuda_stream);

/* Kernel launches of the most recent call on this network. */
int64_t gmco_mlp_last_launch_count(const gmco_mlp *mlp);

/* Text of the most recent network error on the calling host thread. */
const char *gmco_mlp_last_error(void);

/* Warm start with fallback: predicts t for each of the P plans, evaluates the objective of
 * the prediction and of the uniform start (1 s) with the problem's precision, and writes to
 * t0_out (P x n_dwell) the prediction where its objective is not larger, else the uniform
 * start.  from_model[p] (may be NULL) is 1 where the prediction was kept.  t0_out then goes
 * to gmco_solve_batch. */
gmco_status gmco_warm_start(gmco_problem *prob, gmco_mlp *mlp, const float *features,
                            const float *penalty_weights, int64_t P, float t_floor,
                            float *t0_out, int32_t *from_model, void *cuda_stream);

/* Problem sizes as stored (after validation). */
gmco_status gmco_problem_info(const gmco_problem *prob, int64_t *n_pnt, int64_t *n_dwell,
                              int32_t *n_struct, int32_t *precision);

/* Kernel launches made by the most recent solve or evaluate call on this problem. */
int64_t gmco_last_launch_count(const gmco_problem *prob);

/* Steps of the most recent tensor-core solve on this problem whose gradient was formed from
 * the active pairs alone (options.sparse_grad_permille); -1 where the option is off or the
 * form is FP32 (or the count cannot be read). */
int64_t gmco_last_sparse_steps(const gmco_problem *prob);

/* Static description of a status code. */
const char *gmco_status_string(gmco_status s);

/* Text of the most recent error on the calling host thread (empty if none). */
const char *gmco_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
