// Tensor-core (tcgen05, BF16 operands, FP32 accumulate) evaluation path.
#pragma once
#include <cuda.h>

#include <functional>

#include "common.cuh"

namespace gmco {

using AllocFn = std::function<cudaError_t(void **, size_t)>;

constexpr int kTcMaps = 8;
struct TcMaps {
    CUtensorMap m[kTcMaps];
};

// Compact per-evaluation operands of the tensor-core path (cap plan rows).
struct TcBuffers {
    __nv_bfloat16 *T[3] = {nullptr, nullptr, nullptr};   // cap x kpad, split terms of t
    __nv_bfloat16 *dT = nullptr;                         // cap x kpad, t_trial - t (BF16)
    __nv_bfloat16 *G[3] = {nullptr, nullptr, nullptr};   // cap x np_pad, split terms of dF/dd
    float *Wc = nullptr;                                 // cap x n_struct
    int32_t *err = nullptr;  // device flag: nonzero after a pipeline wait gave up
    int32_t cap = 0;
    TcMaps maps1{}, maps2{};   // dose GEMM (A terms, T terms, dT), gradient GEMM (A^T, G)
};

int32_t tc_n_ptiles(const DevProblem &pb);
int32_t tc_max_split(const DevProblem &pb);
SplitPlan tc_split_plan(const DevProblem &pb);
int64_t tc_launches_per_eval();
// MMA products per output element issued by the dose GEMM (which = 1) or gradient GEMM (2).
double tc_mma_units(const DevProblem &pb, bool with_dT, int which);
// Splits A / row_scale into pb->tc_terms BF16 terms (precision 1, 3, 4) or the E4M3 grid
// (precision 2) and builds the transposed copies.  cudaErrorNotSupported when the sizes are
// beyond the tensor-core path (n_dwell > 384 or n_struct > 8).
cudaError_t tc_prepare_problem(DevProblem *pb, int precision, cudaStream_t st,
                               const AllocFn &alloc);
cudaError_t tc_alloc(const DevProblem &pb, int32_t cap, TcBuffers *b, const AllocFn &alloc);
// One evaluation of the compact rows (s.list, s.n_act): prep, dose GEMM + penalty epilogue,
// gradient GEMM, finish.  Writes s.Ft, s.dFt, s.gt.  With dose_out set, the dose GEMM
// writes doses (cap x np_pad FP32) instead of dF/dd and the gradient GEMM is skipped.
cudaError_t tc_launch_eval(const DevProblem &pb, const SolverState &s, const TcBuffers &b,
                           float *Fpart, float *dFpart, float *gpart, int32_t cap, bool with_dT,
                           float *dose_out, bool force_base, cudaStream_t st,
                           int32_t *n_launches, cudaEvent_t *ev = nullptr);
// The trial-row preparation alone (compact rows from s.list / s.n_act).
cudaError_t tc_launch_prep(const DevProblem &pb, const SolverState &s, const TcBuffers &b,
                           int32_t cap, bool force_base, cudaStream_t st);
// The two GEMMs alone, over the compact rows counted by *n_rows (rows written elsewhere).
cudaError_t tc_launch_gemms(const DevProblem &pb, const TcBuffers &b, const int32_t *n_rows,
                            float *Fpart, float *dFpart, float *gpart, int32_t cap, bool with_dT,
                            float *dose_out, cudaStream_t st, int32_t *n_launches,
                            cudaEvent_t *ev = nullptr);

}  // namespace gmco
