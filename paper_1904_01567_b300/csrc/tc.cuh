// Tensor-core (tcgen05, BF16 operands, FP32 accumulate) evaluation path.
//
// The two GEMM kernels work on a list of problems (patients) at once: every problem brings a
// descriptor (row offsets into the shared operand maps, sizes, epilogue buffers), the work
// items of all problems form one list, and each CTA of the persistent grid walks that list.
// A single problem is the list of length one.
#pragma once
#include <cuda.h>

#include <functional>

#include "common.cuh"

namespace gmco {

using AllocFn = std::function<cudaError_t(void **, size_t)>;

constexpr int kMaxMulti = 64;    // problems in one GEMM launch (descriptors in shared memory)
constexpr int kTcActWords = 8;   // active-set counters of a problem (TcDoseProb::act)
constexpr int kTcPrefetch = 6;   // L2 prefetch ranges of a gradient-GEMM launch

// Operand maps.  Dose GEMM: m[0..2] A terms (rows = points, columns = dwells), m[3..5] T terms
// (rows = plans, columns = dwells), m[6], m[7] the two terms of dT.  Gradient GEMM: m[0..2] A^T terms (rows = dwells,
// columns = points), m[3..5] G terms (rows = plans, columns = points).  Problems are stacked
// along the rows of each map.
constexpr int kTcMaps = 8;
struct TcMaps {
    CUtensorMap m[kTcMaps];
};

// Per-problem part of a dose-GEMM launch.
struct TcDoseProb {
    const int32_t *n_rows[2];   // compact-row counters of even and odd steps
    const float4 *pt4;          // np_pad: (D_min, D_max, scale, id) per point
    const int32_t *chunk;       // np_pad / 16: epilogue mode per 16 points
    const float4 *sparams;      // n_struct: (w_min, D_min, D_max, w_max)
    const float *Wc;            // cap x n_struct, w / N_s per compact row
    __nv_bfloat16 *G[3];        // row r at G[j] + r * ld_g: split terms of dF/dd
    float *dose_out;            // row r at dose_out + r * ld_g (dose mode)
    float *Fpart, *dFpart;      // [cap][point tile]
    int32_t a_row;              // first row of this problem's points in the A maps
    int32_t t_row;              // first row of its plans in the T / dT maps
    int32_t kb;                 // K blocks of 64 dwells
    int32_t k16;                // 16-dwell K steps holding data
    int32_t n_ptiles;           // point tiles of 128
    int32_t n_struct;
    int32_t cap;                // plan rows of Fpart / dFpart
    int32_t ld_g;               // row stride of G and dose_out (elements)
    // active-set gradient (single problems; null / 0 otherwise): where the previous step's
    // count of active (plan, point) pairs was at most sp_thr per row of this step, this step
    // writes, instead of the BF16 terms of G, a bit mask of the active points (per row and
    // point tile, 4 words of 32 points) and the FP32 dF/dd of the active pairs only (row r at
    // Gs + r * ld_g, in the units of G)
    uint32_t *mask;             // cap x n_ptiles x 4
    float *Gs;
    int32_t *act;               // [0..1] active-pair counts of even / odd steps, [2..3] the
                                // steps' path (1 = active-set gradient), [4] steps on that path
    int32_t sp_thr;
    int32_t pad2_;
};

// Per-problem part of a gradient-GEMM launch.
struct TcGradProb {
    const int32_t *n_rows[2];
    float *gpart;               // [split][rows][nd_pad]
    SplitPlan sp;               // point splits, from the row count
    int32_t at_row;             // first row of this problem's dwells in the A^T maps
    int32_t g_row;              // first row of its plans in the G maps
    int32_t kb;                 // K blocks of 64 points
    int32_t n_dt;               // dwell tiles of 128 (TMEM lanes)
    int32_t nd_pad;
    const int32_t *act;         // as TcDoseProb::act, or null: a step whose path is the
                                // active-set gradient has no work here
};

// Compact per-evaluation operands of one problem (cap plan rows) and its operand maps.
struct TcBuffers {
    __nv_bfloat16 *T[3] = {nullptr, nullptr, nullptr};   // cap x kpad, split terms of t
    __nv_bfloat16 *dT[2] = {nullptr, nullptr};           // cap x kpad, t_trial - t (two terms)
    __nv_bfloat16 *G[3] = {nullptr, nullptr, nullptr};   // cap x np_pad, split terms of dF/dd
    float *Wc = nullptr;                                 // cap x n_struct
    int32_t *err = nullptr;  // device flag: nonzero after a pipeline wait gave up
    int64_t wait_ns = 1000000000;   // limit of every pipeline wait (gmco_options.wait_limit_us)
    int32_t cap = 0;
    TcMaps maps1{}, maps2{};         // dose GEMM, gradient GEMM
    TcDoseProb *d_dose = nullptr;    // device descriptors of this problem (one each)
    TcGradProb *d_grad = nullptr;
    float *Fpart = nullptr, *dFpart = nullptr, *gpart = nullptr, *dose_out = nullptr;
    SplitPlan sp{};                  // split plan of the gradient GEMM
    int32_t grad_tile = 0;           // plans per gradient-GEMM tile
    uint32_t *mask = nullptr;        // active-set gradient (sparse_permille > 0), see TcDoseProb
    int32_t *act = nullptr;
    float *Gs = nullptr;
    int32_t sp_thr = 0;
    const int32_t *cnt = nullptr;    // the two row counters
};

// Where the trial rows of a problem's compact plans go (tensor-core operand layout).
struct TcRows {
    __nv_bfloat16 *T[3];
    __nv_bfloat16 *dT[2];
    float *Wc;
    int32_t ld;      // row stride of T and dT (elements)
    int32_t kpad;    // row length written (columns past nd_pad are zero)
    int32_t nT;
};

// A GEMM launch over a list of problems.
struct TcLaunchSet {
    TcMaps maps1{}, maps2{};
    const TcDoseProb *dose = nullptr;   // device array of n
    const TcGradProb *grad = nullptr;   // device array of n
    int32_t n = 0;
    int32_t tc_terms = 0;               // BF16 terms of A (all problems alike)
    int64_t max_items1 = 1, max_items2 = 1;   // work items at full capacity (grid bound)
    int32_t grad_tile = 0;              // plans per gradient-GEMM tile (grad_bn of the request)
    // active-set gradient of a single problem (gs_act non-null): its kernel's arguments
    const int32_t *gs_rows[2] = {nullptr, nullptr};
    const uint32_t *gs_mask = nullptr;
    const float *gs_G = nullptr;                                   // dF/dd of the active pairs
    const __nv_bfloat16 *gs_A[3] = {nullptr, nullptr, nullptr};    // A / row_scale terms
    int32_t *gs_act = nullptr;
    float *gs_out = nullptr;                                       // gradient, split 0 of gpart
    int32_t gs_ld = 0, gs_nd = 0, gs_ptiles = 0, gs_kpad = 0, gs_terms = 0, gs_cap = 0;
    // byte ranges the gradient GEMM prefetches into L2 for the update that follows it (the
    // plans' history rows and vectors): that kernel is bound by the MMA issue and leaves DRAM
    // bandwidth to spare, while the update waits on these reads
    const void *pf_ptr[kTcPrefetch] = {};
    int64_t pf_bytes[kTcPrefetch] = {};
    int32_t *err = nullptr;
    int64_t wait_ns = 1000000000;       // limit of every pipeline wait, nanoseconds
};

int32_t tc_n_ptiles(const DevProblem &pb);
int32_t tc_max_split(const DevProblem &pb);
// Default split plan of a problem's gradient GEMM; kb_per_split > 0 fixes the number of
// 64-point blocks per split instead.
SplitPlan tc_split_plan(const DevProblem &pb, int32_t kb_per_split = 0, int32_t grad_tile = 0);
int32_t tc_n_dtiles(const DevProblem &pb);
// Plans per tile of the gradient GEMM: requested 128, or 256 (the default, requested 0 or 256)
// where a stage of 256 fits, else 128.
int grad_bn(int tc_terms, int requested = 0);
int64_t tc_launches_per_eval();
// MMA products per output element issued by the dose GEMM (which = 1) or gradient GEMM (2).
double tc_mma_units(const DevProblem &pb, bool with_dT, int which);
// Splits A / row_scale into pb->tc_terms BF16 terms (precision 1, 3, 4) or the E4M3 grid
// (precision 2) and builds the transposed copies.  cudaErrorNotSupported when the sizes are
// beyond the tensor-core path (n_dwell > 512 or n_struct > 8).
cudaError_t tc_prepare_problem(DevProblem *pb, int precision, cudaStream_t st,
                               const AllocFn &alloc);
// Compact buffers, operand maps and device descriptors of one problem with cap plan rows.
cudaError_t tc_alloc(const DevProblem &pb, int32_t cap, float *Fpart, float *dFpart,
                     float *gpart, float *dose_out, const int32_t *cnt, int32_t split_kb,
                     int32_t grad_tile, int32_t sparse_permille, TcBuffers *b,
                     const AllocFn &alloc);
TcLaunchSet tc_single_set(const DevProblem &pb, const TcBuffers &b);
// Descriptors of one problem inside a launch list: cnt = its two row counters, rows of its
// operands starting at a_row (points, A maps), t_row (plans, T / dT / G maps) and at_row
// (dwells, A^T maps).
TcDoseProb tc_dose_prob(const DevProblem &pb, const int32_t *cnt, const float *Wc,
                        __nv_bfloat16 *const *G, float *dose_out, float *Fpart, float *dFpart,
                        int32_t a_row, int32_t t_row, int32_t cap, int32_t ld_g);
TcGradProb tc_grad_prob(const DevProblem &pb, const int32_t *cnt, float *gpart, SplitPlan sp,
                        int32_t at_row, int32_t g_row);
TcRows tc_rows(const DevProblem &pb, const TcBuffers &b);
// Operand maps over stacked buffers (rows of all problems one after another).
bool tc_encode_map(CUtensorMap *m, const void *ptr, uint64_t cols, uint64_t rows,
                   uint32_t box_cols, uint32_t box_rows);
constexpr int kTcBoxRowsA = 128, kTcBoxRowsT = 128, kTcBoxRowsAT = 128, kTcBoxRowsG = 128;
constexpr int kTcBoxCols = 64;

// One evaluation of the compact rows (s.list, s.n_act): prep, dose GEMM + penalty epilogue,
// gradient GEMM, finish.  Writes s.Ft, s.dFt, s.gt.  With write_dose, the dose GEMM writes
// doses (FP32, the descriptor's dose_out) instead of dF/dd and the gradient GEMM is skipped.
cudaError_t tc_launch_eval(const DevProblem &pb, const SolverState &s, const TcBuffers &b,
                           int32_t cap, bool with_dT, bool write_dose, bool force_base,
                           cudaStream_t st, int32_t *n_launches, cudaEvent_t *ev = nullptr);
// The trial-row preparation alone (compact rows from s.list / s.n_act).
cudaError_t tc_launch_prep(const SolverState &s, const TcRows &r, int32_t cap, bool force_base,
                           cudaStream_t st);
// The two GEMMs over the problems of `set`, each over its compact rows counted by
// n_rows[parity].  zero_next: the dose GEMM also clears every problem's n_rows[parity ^ 1]
// (the next step's counter, which nothing reads during this launch).
cudaError_t tc_launch_gemms(const TcLaunchSet &set, int32_t parity, bool with_dT,
                            bool write_dose, bool zero_next, cudaStream_t st,
                            int32_t *n_launches, cudaEvent_t *ev = nullptr);

}  // namespace gmco
