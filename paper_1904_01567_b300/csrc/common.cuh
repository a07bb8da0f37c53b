// Internal declarations shared by the CUDA translation units of libgmco.
// Device buffers, launch helpers and the solver's per-plan state layout.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "gmco.h"

namespace gmco {

constexpr int kMaxStruct = 16;
constexpr int kMaxHist = 16;
constexpr int kMaxDwell = 1024;

// Per-plan solver state machine (one evaluation per step for every plan not DONE).
enum PlanState : int32_t { ST_INIT = 0, ST_TRIAL = 1, ST_DONE = 2 };

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Problem data resident on the device.
struct DevProblem {
    int64_t n_pnt = 0, n_dwell = 0;
    int64_t np_pad = 0;   // points padded to a multiple of 256 (padding rows of A are 0, sid -1)
    int64_t nd_pad = 0;   // dwells padded to a multiple of 32 (padding columns of A are 0)
    int32_t n_struct = 0;
    float *A32 = nullptr;          // np_pad x nd_pad, Gy/s
    float *row_scale = nullptr;    // np_pad, power-of-two scale of each point's row of A
    int8_t *sid = nullptr;         // np_pad, -1 on padding points
    // tensor-core forms: A / row_scale split into tc_terms BF16 terms, row-major and transposed
    int32_t tc_terms = 0;          // 0 = FP32 SIMT form
    float4 *pt4 = nullptr;         // np_pad: (D_min, D_max, scale, id) per point, dose epilogue
    int32_t *chunk = nullptr;      // np_pad / 16: epilogue mode of each run of 16 points
    int64_t kpad = 0;              // dwells padded to a multiple of 64 (BF16 row length)
    __nv_bfloat16 *Ah[3] = {nullptr, nullptr, nullptr};    // np_pad x kpad
    __nv_bfloat16 *AhT[3] = {nullptr, nullptr, nullptr};   // kpad x np_pad
    float4 *sparams = nullptr;     // n_struct x (w_min, D_min, D_max, w_max)
    float *inv_count = nullptr;    // n_struct, 1 / N_s
};

// Point splits of a gradient GEMM, chosen at run time from the number of rows so that a small
// batch still spreads over the SMs.  Shared by the GEMM kernels and the kernels that read
// their partial sums, which must agree on it.
struct SplitPlan {
    int32_t rows_per_tile;   // plan rows per CTA tile
    int32_t other_tiles;     // CTA tiles along the output columns
    int32_t kb_total;        // K blocks (of points) in total
    int32_t target_ctas;     // CTAs to aim for
    int32_t max_split;       // grid extent along the split dimension
    int32_t min_kb;          // fewest K blocks per split: bounds the partial sums a reader adds
};

__host__ __device__ inline void split_plan(const SplitPlan &p, int32_t n_rows, int32_t *kbps,
                                           int32_t *n_split)
{
    int32_t tiles = (n_rows + p.rows_per_tile - 1) / p.rows_per_tile;
    tiles = (tiles < 1 ? 1 : tiles) * (p.other_tiles < 1 ? 1 : p.other_tiles);
    int32_t target = p.target_ctas / tiles;
    target = target < 1 ? 1 : (target > p.max_split ? p.max_split : target);
    int32_t k = (p.kb_total + target - 1) / target;
    k = k < p.min_kb ? p.min_kb : k;
    *kbps = k;
    *n_split = (p.kb_total + k - 1) / k;
}

// Buffers of one evaluation pass over `rows` compact plan rows.
struct EvalArgs {
    DevProblem pb;           // by value: kernels read the problem's pointers and sizes
    const int32_t *n_rows;   // device scalar: number of valid compact rows
    int32_t cap;             // allocated compact rows
    const float *Tt;         // cap x nd_pad trial dwell times
    const float *dT;         // cap x nd_pad change of dwell times vs the base point, or null
    const float *Wc;         // cap x n_struct, w_ps / N_s
    float *G;                // cap x np_pad, dF/dd per point (mode G) or dose (mode D)
    float *Fpart;            // cap x n_ptiles, per point tile partial of F (a row's contiguous)
    float *dFpart;           // cap x n_ptiles, partial of F(trial) - F(base)
    float *gpart;            // n_split x rows x nd_pad, partial of A^T G (rows = *n_rows)
    SplitPlan sp;            // split plan of the gradient GEMM that wrote gpart
};

// Plan-indexed solver state (capacity P).
struct SolverState {
    int32_t P = 0, m = 10, nd_pad = 0, n_struct = 0;
    float *x = nullptr, *g = nullptr, *p = nullptr, *xt = nullptr, *gt = nullptr;  // P x nd_pad
    float *S = nullptr, *Y = nullptr;   // P x m x nd_pad
    double *rho = nullptr;              // P x m
    double *gamma = nullptr;            // P
    double *F = nullptr, *Ft = nullptr, *dFt = nullptr, *gtp = nullptr, *alpha = nullptr;
    int32_t *state = nullptr, *status = nullptr, *iters = nullptr, *maxit = nullptr;
    int32_t *ls = nullptr, *hcount = nullptr, *hnewest = nullptr;
    int32_t *nsmall = nullptr;          // consecutive iterations below the stop tolerance
    int32_t *nevals = nullptr;          // objective evaluations so far
    int32_t *slot_of = nullptr;         // compact row of each plan in the current evaluation
    int32_t *cnt = nullptr;             // 2 counters: rows of even and odd steps
    float *Wn = nullptr;                // P x n_struct, w / N_s
    int32_t *list = nullptr;            // compact row -> plan
    int32_t *n_act = nullptr;           // device scalar
    int32_t *n_live = nullptr;          // device scalar: plans not DONE after the last update
};

// Inputs of a fused solver step: the evaluation's partial sums and where the next step's
// compact rows go.
struct StepArgs {
    const float *Fpart, *dFpart;     // cap x n_ptiles
    const float *gpart;              // n_split x rows x nd_pad
    int32_t n_ptiles, cap;
    SplitPlan sp;
    const int32_t *sp_flag;          // nonzero: this step's gradient is split 0 alone (the
                                     // active-set gradient); null or zero: the split plan
    const int32_t *rows_cur;         // rows evaluated this step
    int32_t *rows_next;              // slot counter of the next step
    int32_t fmt;                     // 0: FP32 rows (Tc, dTc), 1: BF16 split rows (Tb, dTb)
    float *Tc, *dTc;
    __nv_bfloat16 *Tb[3];
    __nv_bfloat16 *dTb[2];
    int32_t nT, kpad;                // BF16 terms of t; row length written (columns >= nd_pad zero)
    int32_t ldT;                     // row stride of Tb / dTb (elements)
    float *Wc;
};

// A problem's part of a multi-problem solver step: its state and its step arguments.
struct StepDesc {
    SolverState s;
    StepArgs a;
};

struct UpdateParams {
    double c1, tol;
    int32_t max_ls;
    int32_t stop_window;
    int32_t max_evals;               // evaluations per plan, 0 = no limit
};

// ---- launchers (return cudaError_t of the launch) ----
cudaError_t launch_solver_init(const SolverState &s, const DevProblem &pb, const float *W,
                               const float *t0, int32_t max_iters, cudaStream_t st);
cudaError_t launch_compact(const SolverState &s, int32_t mode, cudaStream_t st);
cudaError_t launch_prep_fp32(const SolverState &s, const DevProblem &pb, float *Tc, float *dTc,
                             float *Wc, bool force_base, cudaStream_t st);
cudaError_t launch_finish(const SolverState &s, const EvalArgs &e, int32_t n_ptiles,
                          cudaStream_t st);
cudaError_t launch_step(const SolverState &s, const UpdateParams &u, const StepArgs &a,
                        cudaStream_t st);
// The step of every plan of n problems: blocks [block_start[p], block_start[p+1]) take the
// plans of problem p (8 per block); d[p] holds its state and step arguments.
cudaError_t launch_step_multi(const StepDesc *d, const int32_t *block_start, int32_t n,
                              int32_t total_blocks, int32_t max_nd_pad, const UpdateParams &u,
                              cudaStream_t st);
// *sum = sum over p < n of *counters[p].
cudaError_t launch_sum_counters(int32_t *const *counters, int32_t n, int32_t *sum, cudaStream_t st);
// Dose rate matrix (doserate.cu): src = Lambda, S_K, unit factor, r_min, g0, g1, g2; *bad is
// set to 1 where g(r) <= 0.  n_dwell <= 1024.
cudaError_t launch_dose_rate(const float *pts, int64_t n_pnt, const float *dw, int32_t n_dwell,
                             const double *src, float *A, int32_t *bad, cudaStream_t st);
// Plan pool (pool.cu): RTOG classes and the selected plan of P DVH rows (crit: 6 values, see
// gmco_rtog); non-dominated flags of P objective rows of K <= 16 values (all minimised).
cudaError_t launch_rtog(const float *dvh, int64_t P, const double *crit, int32_t *cls, int32_t *selected,
                        cudaStream_t st);
cudaError_t launch_pareto(const double *obj, int64_t P, int32_t K, int32_t *nondom, cudaStream_t st);
// Annealing engine (sa.cu): moved weights x = xc + delta (2u - 1) of iteration k, and the
// Metropolis decision on their objectives Ft (k < 0: the start point's evaluation).
cudaError_t launch_sa_propose(float *x, const float *xc, int64_t P, int64_t nd, int64_t nd_pad,
                              uint64_t seed, int32_t k, double delta, cudaStream_t st);
cudaError_t launch_sa_accept(const float *x, float *xc, float *xb, int64_t P, int64_t nd_pad,
                             const double *Ft, double *Fc, double *Fb, double *F0, int32_t *acc,
                             uint64_t seed, int32_t k, double temp, cudaStream_t st);
cudaError_t launch_count_live(const SolverState &s, cudaStream_t st);
cudaError_t launch_reopen(const SolverState &s, int32_t extra_iters, cudaStream_t st);
cudaError_t launch_profile_setup(const SolverState &s, cudaStream_t st);
cudaError_t launch_square(const float *x, float *t, int64_t rows, int64_t nd, int64_t nd_pad,
                          cudaStream_t st);

// SIMT FP32 evaluation
enum EvalMode : int32_t { MODE_G = 0, MODE_DOSE = 1 };
int32_t simt_n_ptiles(const DevProblem &pb);
SplitPlan simt_split_plan(const DevProblem &pb);
cudaError_t launch_gemm1_simt(const EvalArgs &e, int32_t mode, cudaStream_t st);
cudaError_t launch_gemm2_simt(const EvalArgs &e, cudaStream_t st);

// Allocation-free FP32 evaluation (noalloc.cu): scratch in a fixed device array.
size_t noalloc_scratch_bytes();
size_t noalloc_required_bytes(const DevProblem &pb, int64_t P);
cudaError_t noalloc_evaluate(const DevProblem &pb, const float *W, int64_t P, const float *X,
                             double *F, float *grad, cudaStream_t st);

// Dose calculation points of the analytic structures (points.cu): geo = a, b, c, urethra_r,
// rectum_r, rectum_y, rectum_half_len, bladder_r, bladder_z; counts[4] per structure; writes
// structure-major points (x, y, z) and ids to device buffers.  *short_struct = the structure
// whose candidates ran out (or -1).  Synchronises st.
cudaError_t sample_points_dev(const double *geo, const int64_t *counts, uint64_t seed, float *pts,
                              int32_t *sid, cudaStream_t st, int32_t *short_struct);

// DVH indices of P dose rows (P x np_pad, row stride ld)
cudaError_t launch_dvh(const DevProblem &pb, const float *D, int64_t ld, const int32_t *rows,
                       int32_t P, double rx, float *dvh_out, cudaStream_t st);

}  // namespace gmco
