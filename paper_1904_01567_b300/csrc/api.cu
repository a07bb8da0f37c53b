// Host side of the C ABI declared in include/gmco.h: argument validation, device residency
// of the problem, the solver workspace, the graph-captured step loop and result copies.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

using namespace gmco;

namespace {

thread_local std::string g_last_error;

void set_error(const char *what, cudaError_t e)
{
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    g_last_error = buf;
}

void set_error_msg(const char *what) { g_last_error = what; }

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) {                                   \
            set_error(#call, e_);                                  \
            return (e_ == cudaErrorMemoryAllocation) ? GMCO_ENOMEM \
                                                     : GMCO_ECUDA; \
        }                                                          \
    } while (0)

#define CKS(expr)                       \
    do {                                \
        gmco_status s_ = (expr);        \
        if (s_ != GMCO_OK) return s_;   \
    } while (0)

// Every device allocation of a problem is registered here and freed with it.
struct DevArena {
    std::vector<void *> ptrs;
    template <class T>
    cudaError_t alloc(T **p, size_t count)
    {
        *p = nullptr;
        if (count == 0) count = 1;
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, count * sizeof(T));
        if (e != cudaSuccess) return e;
        ptrs.push_back(q);
        *p = static_cast<T *>(q);
        return cudaSuccess;
    }
    void release()
    {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

__global__ void k_count_bad(const float *v, int64_t n, int32_t allow_negative, int32_t *bad)
{
    int c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float x = v[i];
        if (!isfinite(x) || (!allow_negative && x < 0.0f)) ++c;
    }
    if (c) atomicAdd(bad, c);
}

}  // namespace

// Compact rows of P plans at given dwell times T (P x nd, s): row i = plan i, t padded with
// zeros to nd_pad, weights zero (only doses are formed from these rows).
__global__ void k_rows_from_times(const float *__restrict__ T, int32_t P, int32_t nd, int32_t nd_pad,
                                  int32_t S, float *__restrict__ Tc, float *__restrict__ Wc,
                                  int32_t *__restrict__ list, int32_t *__restrict__ n_act)
{
    const int i = blockIdx.x;
    if (i >= P) return;
    for (int l = threadIdx.x; l < nd_pad; l += blockDim.x)
        Tc[(size_t)i * nd_pad + l] = l < nd ? T[(size_t)i * nd + l] : 0.0f;
    if (threadIdx.x < S) Wc[(size_t)i * S + threadIdx.x] = 0.0f;
    if (threadIdx.x == 0) {
        list[i] = i;
        if (i == 0) *n_act = P;
    }
}

struct gmco_problem {
    int device = 0;
    gmco_options opt{};
    DevProblem pb{};
    std::vector<int64_t> counts;
    DevArena arena;      // problem data
    DevArena ws_arena;   // workspace, re-created when the batch capacity grows
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int32_t *d_flag = nullptr;   // validation counter
    int32_t *h_pinned = nullptr; // pinned host scalars

    // workspace (capacity cap plans)
    int32_t cap = 0;
    SolverState s{};
    float *Tc = nullptr, *dTc = nullptr, *Wc = nullptr, *G = nullptr;
    float *Fpart = nullptr, *dFpart = nullptr, *gpart = nullptr;
    int32_t n_ptiles = 1;
    TcBuffers tcb{};
    float *dW = nullptr, *dT0 = nullptr, *dTout = nullptr, *dDvh = nullptr;
    double *dObj = nullptr;
    int32_t *dIters = nullptr, *dStatus = nullptr;
    float *dDose = nullptr;
    int64_t dose_cap = 0;

    // cached step graphs, one per evaluation form
    struct GraphKey {
        int32_t P = -1, form = -1, max_ls = -1, steps = -1, window = -1, max_evals = -1;
        double tol = -1, c1 = -1;
        bool operator==(const GraphKey &o) const
        {
            return P == o.P && form == o.form && max_ls == o.max_ls && steps == o.steps &&
                   window == o.window && max_evals == o.max_evals && tol == o.tol && c1 == o.c1;
        }
    };
    GraphKey gkey[2];
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};

    int64_t launches = 0;
    int64_t ws_gen = 0;   // incremented whenever the workspace is re-created
};

namespace {

gmco_status count_bad(gmco_problem *pr, const float *dv, int64_t n, bool allow_negative,
                      int32_t *out)
{
    CK(cudaMemsetAsync(pr->d_flag, 0, sizeof(int32_t), pr->stream));
    if (n > 0) {
        const int blocks = (int)std::min<int64_t>(ceil_div(n, 256), 148 * 8);
        k_count_bad<<<blocks, 256, 0, pr->stream>>>(dv, n, allow_negative ? 1 : 0, pr->d_flag);
        CK(cudaGetLastError());
        pr->launches++;
    }
    CK(cudaMemcpyAsync(pr->h_pinned, pr->d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost,
                       pr->stream));
    CK(cudaStreamSynchronize(pr->stream));
    *out = pr->h_pinned[0];
    return GMCO_OK;
}

void destroy_graphs(gmco_problem *pr)
{
    for (int k = 0; k < 2; ++k) {
        if (pr->gexec[k]) cudaGraphExecDestroy(pr->gexec[k]);
        pr->gexec[k] = nullptr;
        pr->gkey[k] = gmco_problem::GraphKey{};
    }
}

// Largest number of gradient-partial rows (splits x rows) any row count up to cap can use.
int64_t max_split_rows(const SplitPlan &sp, int32_t cap)
{
    int64_t best = 0;
    for (int32_t n = 1; n <= cap; ++n) {
        int32_t kbps, ns;
        split_plan(sp, n, &kbps, &ns);
        best = std::max<int64_t>(best, (int64_t)ns * n);
    }
    return best;
}

gmco_status ensure_workspace(gmco_problem *pr, int32_t P)
{
    if (P <= pr->cap) return GMCO_OK;
    CK(cudaStreamSynchronize(pr->stream));
    destroy_graphs(pr);
    pr->ws_arena.release();
    pr->cap = 0;
    const DevProblem &pb = pr->pb;
    const int32_t cap = std::max<int32_t>(P, 8);
    const int32_t m = pr->opt.m, nd = (int32_t)pb.nd_pad, S = pb.n_struct;
    DevArena &a = pr->ws_arena;
    SolverState &s = pr->s;
    s = SolverState{};
    s.P = cap;
    s.m = m;
    s.nd_pad = nd;
    s.n_struct = S;
    const size_t vn = (size_t)cap * nd;
    CK(a.alloc(&s.x, vn)); CK(a.alloc(&s.g, vn)); CK(a.alloc(&s.p, vn));
    CK(a.alloc(&s.xt, vn)); CK(a.alloc(&s.gt, vn));
    CK(a.alloc(&s.S, vn * m)); CK(a.alloc(&s.Y, vn * m));
    CK(a.alloc(&s.rho, (size_t)cap * m)); CK(a.alloc(&s.gamma, (size_t)cap));
    CK(a.alloc(&s.F, (size_t)cap)); CK(a.alloc(&s.Ft, (size_t)cap));
    CK(a.alloc(&s.dFt, (size_t)cap)); CK(a.alloc(&s.gtp, (size_t)cap));
    CK(a.alloc(&s.alpha, (size_t)cap));
    CK(a.alloc(&s.state, (size_t)cap)); CK(a.alloc(&s.status, (size_t)cap));
    CK(a.alloc(&s.iters, (size_t)cap)); CK(a.alloc(&s.maxit, (size_t)cap));
    CK(a.alloc(&s.ls, (size_t)cap)); CK(a.alloc(&s.hcount, (size_t)cap));
    CK(a.alloc(&s.hnewest, (size_t)cap)); CK(a.alloc(&s.nsmall, (size_t)cap));
    CK(a.alloc(&s.nevals, (size_t)cap));
    CK(a.alloc(&s.slot_of, (size_t)cap)); CK(a.alloc(&s.cnt, 2));
    CK(a.alloc(&s.Wn, (size_t)cap * S));
    CK(a.alloc(&s.list, (size_t)cap)); CK(a.alloc(&s.n_live, 1));
    s.n_act = s.cnt;   // the compaction's row count is the even-step counter
    CK(cudaMemset(s.S, 0, vn * m * sizeof(float)));
    CK(cudaMemset(s.Y, 0, vn * m * sizeof(float)));

    pr->n_ptiles = simt_n_ptiles(pb);
    CK(a.alloc(&pr->Tc, vn)); CK(a.alloc(&pr->dTc, vn)); CK(a.alloc(&pr->Wc, (size_t)cap * S));
    CK(a.alloc(&pr->G, (size_t)cap * pb.np_pad));
    const int32_t nparts = std::max(pr->n_ptiles, tc_n_ptiles(pb));
    CK(a.alloc(&pr->Fpart, (size_t)nparts * cap));
    CK(a.alloc(&pr->dFpart, (size_t)nparts * cap));
    int64_t grows = max_split_rows(simt_split_plan(pb), cap);
    if (pr->opt.precision != GMCO_PREC_FP32)
        grows = std::max(grows, max_split_rows(tc_split_plan(pb, pr->opt.grad_split_kb, pr->opt.grad_plan_tile), cap));
    CK(a.alloc(&pr->gpart, (size_t)grows * pb.nd_pad));
    if (pr->opt.precision != GMCO_PREC_FP32) {
        cudaError_t e = tc_alloc(pb, cap, pr->Fpart, pr->dFpart, pr->gpart, pr->G, s.cnt,
                                 pr->opt.grad_split_kb, pr->opt.grad_plan_tile,
                                 pr->opt.sparse_grad_permille, &pr->tcb, [&](void **p, size_t bytes) {
                                     unsigned char *q = nullptr;
                                     cudaError_t r = a.alloc(&q, bytes);
                                     *p = q;
                                     return r;
                                 });
        CK(e);
        pr->tcb.wait_ns = (int64_t)pr->opt.wait_limit_us * 1000;
    }
    CK(a.alloc(&pr->dW, (size_t)cap * S));
    CK(a.alloc(&pr->dT0, (size_t)cap * pb.n_dwell));
    CK(a.alloc(&pr->dTout, (size_t)cap * pb.n_dwell));
    CK(a.alloc(&pr->dDvh, (size_t)cap * GMCO_DVH_K));
    CK(a.alloc(&pr->dObj, (size_t)cap));
    CK(a.alloc(&pr->dIters, (size_t)cap));
    CK(a.alloc(&pr->dStatus, (size_t)cap));
    pr->dDose = nullptr;
    pr->dose_cap = 0;
    pr->cap = cap;
    pr->ws_gen++;
    return GMCO_OK;
}

// Launches one evaluation of every compact row (rows from s.list / s.n_act) in `form`
// (0 = FP32 SIMT, 1 = tensor-core BF16) with F, dF and the gradient.
gmco_status launch_eval(gmco_problem *pr, SolverState s, int form, bool with_dT,
                        cudaStream_t st, cudaEvent_t *ev = nullptr)
{
    const DevProblem &pb = pr->pb;
    if (form == 0) {
        if (ev) CK(cudaEventRecord(ev[0], st));
        CK(launch_prep_fp32(s, pb, pr->Tc, with_dT ? pr->dTc : nullptr, pr->Wc, false, st));
        if (ev) CK(cudaEventRecord(ev[1], st));
        EvalArgs e{};
        e.pb = pb;
        e.n_rows = s.n_act;
        e.cap = pr->cap;
        e.Tt = pr->Tc;
        e.dT = with_dT ? pr->dTc : nullptr;
        e.Wc = pr->Wc;
        e.G = pr->G;
        e.Fpart = pr->Fpart;
        e.dFpart = pr->dFpart;
        e.gpart = pr->gpart;
        e.sp = simt_split_plan(pb);
        CK(launch_gemm1_simt(e, MODE_G, st));
        if (ev) CK(cudaEventRecord(ev[2], st));
        CK(launch_gemm2_simt(e, st));
        if (ev) CK(cudaEventRecord(ev[3], st));
        CK(launch_finish(s, e, pr->n_ptiles, st));
        if (ev) CK(cudaEventRecord(ev[4], st));
        pr->launches += 4;
    } else {
        int32_t nl = 0;
        CK(tc_launch_eval(pb, s, pr->tcb, pr->cap, with_dT, false, false, st, &nl, ev));
        pr->launches += nl;
    }
    return GMCO_OK;
}

// Dose-mode FP32 evaluation of every plan at x: doses into pr->G (rows = plans in list
// order), objectives into s.Ft.
gmco_status launch_dose_eval(gmco_problem *pr, const SolverState &s, cudaStream_t st)
{
    const DevProblem &pb = pr->pb;
    CK(launch_compact(s, 1, st));
    CK(launch_prep_fp32(s, pb, pr->Tc, nullptr, pr->Wc, true, st));
    EvalArgs e{};
    e.pb = pb;
    e.n_rows = s.n_act;
    e.cap = pr->cap;
    e.Tt = pr->Tc;
    e.dT = nullptr;
    e.Wc = pr->Wc;
    e.G = pr->G;
    e.Fpart = pr->Fpart;
    e.dFpart = nullptr;
    e.gpart = nullptr;
    e.sp = simt_split_plan(pb);
    CK(launch_gemm1_simt(e, MODE_DOSE, st));
    CK(launch_finish(s, e, pr->n_ptiles, st));
    pr->launches += 4;
    return GMCO_OK;
}

// One solver step = the form's dose and gradient GEMMs over this step's compact rows, the
// reset of the next step's row counter, and the fused update (k_step) that writes the next
// step's rows.  Step k uses counter k % 2; `steps` is even so a graph starts on counter 0.
gmco_status record_steps(gmco_problem *pr, int form, int steps, const UpdateParams &u,
                         int32_t P, cudaStream_t st)
{
    SolverState s = pr->s;
    const DevProblem &pb = pr->pb;
    for (int k = 0; k < steps; ++k) {
        int32_t *cur = s.cnt + (k & 1), *next = s.cnt + ((k + 1) & 1);
        StepArgs a{};
        a.Fpart = pr->Fpart;
        a.dFpart = pr->dFpart;
        a.gpart = pr->gpart;
        a.cap = pr->cap;
        a.rows_cur = cur;
        a.rows_next = next;
        if (form == 0) {
            EvalArgs e{};
            e.pb = pb;
            e.n_rows = cur;
            e.cap = pr->cap;
            e.Tt = pr->Tc;
            e.dT = pr->dTc;
            e.Wc = pr->Wc;
            e.G = pr->G;
            e.Fpart = pr->Fpart;
            e.dFpart = pr->dFpart;
            e.gpart = pr->gpart;
            e.sp = simt_split_plan(pb);
            CK(launch_gemm1_simt(e, MODE_G, st));
            CK(launch_gemm2_simt(e, st));
            a.n_ptiles = pr->n_ptiles;
            a.sp = e.sp;
            a.fmt = 0;
            a.Tc = pr->Tc;
            a.dTc = pr->dTc;
            a.Wc = pr->Wc;
        } else {
            // the dose GEMM also clears the next step's counter
            int32_t nl = 0;
            // the update that follows reads the plans' history rows and vectors: the gradient
            // GEMM brings them into L2
            TcLaunchSet set = tc_single_set(pb, pr->tcb);
            const int64_t vbytes = (int64_t)P * pb.nd_pad * (int64_t)sizeof(float);
            const void *ranges[kTcPrefetch] = {s.S, s.Y, s.x, s.p, s.g, s.xt};
            const int64_t sizes[kTcPrefetch] = {vbytes * s.m, vbytes * s.m, vbytes, vbytes, vbytes, vbytes};
            for (int r = 0; r < kTcPrefetch; ++r) {
                set.pf_ptr[r] = ranges[r];
                set.pf_bytes[r] = sizes[r];
            }
            CK(tc_launch_gemms(set, k & 1, true, false, true, st, &nl));
            a.n_ptiles = tc_n_ptiles(pb);
            a.sp = pr->tcb.sp;
            a.sp_flag = pr->tcb.act ? pr->tcb.act + 2 + (k & 1) : nullptr;
            a.fmt = 1;
            for (int j = 0; j < 3; ++j) a.Tb[j] = pr->tcb.T[j];
            a.dTb[0] = pr->tcb.dT[0];
            a.dTb[1] = pr->tcb.dT[1];
            a.nT = std::max(pb.tc_terms, 2);
            a.kpad = (int32_t)pb.kpad;
            a.ldT = (int32_t)pb.kpad;
            a.Wc = pr->tcb.Wc;
        }
        if (form == 0) CK(cudaMemsetAsync(next, 0, sizeof(int32_t), st));
        CK(launch_step(s, u, a, st));
    }
    return GMCO_OK;
}

// Runs the step loop with evaluation `form` until every plan is DONE.
gmco_status check_tc_error(gmco_problem *pr);

gmco_status run_loop(gmco_problem *pr, int form, int32_t P, const UpdateParams &u,
                     int64_t max_steps, int64_t *steps_done)
{
    const int steps = (int)round_up(std::max(2, pr->opt.steps_per_poll), 2);
    // rows of the first step: every plan in INIT or TRIAL, by compaction and preparation
    {
        SolverState s0 = pr->s;
        if (form != 0 && pr->tcb.act) {
            // active-set counters: the first step reads a count above any threshold (dense)
            CK(cudaMemsetAsync(pr->tcb.act, 0, kTcActWords * sizeof(int32_t), pr->stream));
            CK(cudaMemsetAsync(pr->tcb.act + 1, 0x7f, sizeof(int32_t), pr->stream));
        }
        CK(launch_compact(s0, 0, pr->stream));
        if (form == 0) {
            CK(launch_prep_fp32(s0, pr->pb, pr->Tc, pr->dTc, pr->Wc, false, pr->stream));
        } else {
            CK(tc_launch_prep(s0, tc_rows(pr->pb, pr->tcb), pr->cap, false, pr->stream));
        }
        pr->launches += 2;
    }
    gmco_problem::GraphKey key;
    key.P = P;
    key.form = form;
    key.max_ls = u.max_ls;
    key.steps = steps;
    key.window = u.stop_window;
    key.max_evals = u.max_evals;
    key.tol = u.tol;
    key.c1 = u.c1;
    if (!(pr->gkey[form] == key) || !pr->gexec[form]) {
        if (pr->gexec[form]) cudaGraphExecDestroy(pr->gexec[form]);
        pr->gexec[form] = nullptr;
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(pr->stream, cudaStreamCaptureModeThreadLocal));
        const int64_t l0 = pr->launches;
        gmco_status rs = record_steps(pr, form, steps, u, P, pr->stream);
        pr->launches = l0;
        cudaError_t ee = cudaStreamEndCapture(pr->stream, &g);
        if (rs != GMCO_OK) {
            if (g) cudaGraphDestroy(g);
            return rs;
        }
        CK(ee);
        cudaError_t ei = cudaGraphInstantiate(&pr->gexec[form], g, 0);
        cudaGraphDestroy(g);
        CK(ei);
        pr->gkey[form] = key;
    }
    // launches per graph: steps x (dose GEMM + gradient GEMM [+ active-set gradient] + k_step);
    // memsets not counted
    const int64_t per_graph = (int64_t)steps * (form != 0 && pr->tcb.act ? 4 : 3);
    int64_t done = 0;
    for (;;) {
        CK(cudaGraphLaunch(pr->gexec[form], pr->stream));
        pr->launches += per_graph;
        done += steps;
        CK(cudaMemcpyAsync(pr->h_pinned, pr->s.n_act, sizeof(int32_t), cudaMemcpyDeviceToHost,
                           pr->stream));
        if (form != 0 && pr->tcb.err)
            CK(cudaMemcpyAsync(pr->h_pinned + 1, pr->tcb.err, sizeof(int32_t),
                               cudaMemcpyDeviceToHost, pr->stream));
        CK(cudaStreamSynchronize(pr->stream));
        if (form != 0 && pr->tcb.err && pr->h_pinned[1] != 0) {
            // a pipeline wait gave up: stop stepping; check_tc_error reports and clears it
            *steps_done = done;
            return check_tc_error(pr);
        }
        if (pr->h_pinned[0] == 0) break;
        if (done >= max_steps) {
            *steps_done = done;
            return GMCO_ETIMEOUT;
        }
    }
    *steps_done = done;
    return GMCO_OK;
}

// A tensor-core pipeline wait that gave up (never expected) leaves a code in tcb.err.
gmco_status check_tc_error(gmco_problem *pr)
{
    if (!pr->tcb.err) return GMCO_OK;
    CK(cudaMemcpyAsync(pr->h_pinned + 1, pr->tcb.err, sizeof(int32_t), cudaMemcpyDeviceToHost,
                       pr->stream));
    CK(cudaStreamSynchronize(pr->stream));
    if (pr->h_pinned[1] != 0) {
        char buf[128];
        snprintf(buf, sizeof buf, "tensor-core pipeline wait timed out (code %d)", pr->h_pinned[1]);
        set_error_msg(buf);
        cudaMemsetAsync(pr->tcb.err, 0, sizeof(int32_t), pr->stream);
        return GMCO_ECUDA;
    }
    return GMCO_OK;
}

gmco_status stage_in(gmco_problem *pr, const void *src, void *dst, size_t bytes)
{
    if (bytes == 0) return GMCO_OK;
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, pr->stream));
    return GMCO_OK;
}

gmco_status begin_call(gmco_problem *pr, void *user_stream)
{
    CK(cudaSetDevice(pr->device));
    CK(cudaEventRecord(pr->ev_in, (cudaStream_t)user_stream));
    CK(cudaStreamWaitEvent(pr->stream, pr->ev_in, 0));
    return GMCO_OK;
}

gmco_status end_call(gmco_problem *pr, void *user_stream)
{
    CK(cudaEventRecord(pr->ev_out, pr->stream));
    CK(cudaStreamWaitEvent((cudaStream_t)user_stream, pr->ev_out, 0));
    CK(cudaStreamSynchronize(pr->stream));
    return GMCO_OK;
}


// Start of each plan: the model's prediction where its objective is not larger than the
// uniform start's (a NaN objective selects the uniform start), else t = 1 s.
__global__ void k_choose_start(const double *__restrict__ F_pred, const double *__restrict__ F_unif,
                               const float *__restrict__ t_pred, int64_t nd, float *__restrict__ t0,
                               int32_t *__restrict__ flag)
{
    const int64_t p = blockIdx.x;
    const bool use = F_pred[p] <= F_unif[p];
    for (int64_t l = threadIdx.x; l < nd; l += blockDim.x) t0[p * nd + l] = use ? t_pred[p * nd + l] : 1.0f;
    if (threadIdx.x == 0) flag[p] = use ? 1 : 0;
}

}  // namespace

// ------------------------------------------------------------------ several patients
struct gmco_multi {
    int device = 0;
    std::vector<gmco_problem *> probs;
    int32_t n = 0;
    int32_t tc_terms = 0;
    int32_t split_kb = 16;
    int32_t grad_tile = 0;         // plans per gradient-GEMM tile (0 = the precision's default)
    gmco_options opt{};
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int32_t *h_pinned = nullptr;
    DevArena arena;   // stacked BF16 terms of A and A^T (for the life of the object)
    DevArena ws;      // per-batch buffers, re-created when the batch shape changes
    __nv_bfloat16 *Ah[3] = {nullptr, nullptr, nullptr}, *AhT[3] = {nullptr, nullptr, nullptr};
    int64_t kpad_max = 0, np_max = 0, rows_A = 0, rows_AT = 0;
    int32_t max_nd_pad = 0;
    std::vector<int64_t> a_row, at_row;
    int32_t *err = nullptr;
    // workspace of the current batch shape
    std::vector<int64_t> caps, gens;
    int32_t ws_split = -1, ws_tile = -1;
    std::vector<int64_t> t_row;
    std::vector<SolverState> st;   // each patient's state, P = its plans
    __nv_bfloat16 *T[3] = {nullptr, nullptr, nullptr}, *dT[2] = {nullptr, nullptr};
    __nv_bfloat16 *G[3] = {nullptr, nullptr, nullptr};
    float *Wc = nullptr;
    std::vector<float *> Wc_p;
    TcLaunchSet set;
    StepDesc *d_step = nullptr;    // 2n: parity 0, then parity 1
    int32_t *d_block_start = nullptr;
    int32_t total_blocks = 0;
    int32_t **d_cnt = nullptr;
    int32_t *d_sum = nullptr;
    // cached step graph
    std::vector<int64_t> gkey_caps;
    int32_t gkey_split = -1, gkey_steps = -1, gkey_tile = -1;
    double gkey_tol = -1.0;
    cudaGraphExec_t gexec = nullptr;
    int64_t launches = 0;
};

namespace {

void multi_destroy_graph(gmco_multi *m)
{
    if (m->gexec) cudaGraphExecDestroy(m->gexec);
    m->gexec = nullptr;
    m->gkey_caps.clear();
}

// Stacked per-batch buffers, descriptors and operand maps for P[p] plans per patient.
gmco_status multi_workspace(gmco_multi *m, const std::vector<int64_t> &P)
{
    std::vector<int64_t> gens((size_t)m->n);
    for (int p = 0; p < m->n; ++p) {
        CKS(ensure_workspace(m->probs[p], (int32_t)P[p]));
        gens[p] = m->probs[p]->ws_gen;
    }
    if (m->caps == P && m->gens == gens && m->ws_split == m->split_kb && m->ws_tile == m->grad_tile)
        return GMCO_OK;
    CK(cudaStreamSynchronize(m->stream));
    multi_destroy_graph(m);
    m->ws.release();
    m->caps.clear();
    const int n = m->n;
    const int nT = std::max(m->tc_terms, 2);
    DevArena &a = m->ws;
    m->t_row.assign((size_t)n, 0);
    int64_t R = 0, wsum = 0;
    for (int p = 0; p < n; ++p) {
        m->t_row[p] = R;
        R += P[p];
        wsum += P[p] * m->probs[p]->pb.n_struct;
    }
    for (int j = 0; j < nT; ++j) {
        CK(a.alloc(&m->T[j], (size_t)R * m->kpad_max));
        CK(a.alloc(&m->G[j], (size_t)R * m->np_max));
        CK(cudaMemset(m->T[j], 0, (size_t)R * m->kpad_max * 2));
        CK(cudaMemset(m->G[j], 0, (size_t)R * m->np_max * 2));
    }
    for (int j = 0; j < 2; ++j) {
        CK(a.alloc(&m->dT[j], (size_t)R * m->kpad_max));
        CK(cudaMemset(m->dT[j], 0, (size_t)R * m->kpad_max * 2));
    }
    CK(a.alloc(&m->Wc, (size_t)wsum));
    bool ok = true;
    TcLaunchSet &set = m->set;
    set = TcLaunchSet{};
    set.grad_tile = grad_bn(m->tc_terms, m->grad_tile);
    for (int i = 0; i < m->tc_terms; ++i) {
        ok = ok && tc_encode_map(&set.maps1.m[i], m->Ah[i], m->kpad_max, m->rows_A, kTcBoxCols, kTcBoxRowsA);
        ok = ok && tc_encode_map(&set.maps2.m[i], m->AhT[i], m->np_max, m->rows_AT, kTcBoxCols, kTcBoxRowsAT);
    }
    for (int j = 0; j < nT; ++j) {
        ok = ok && tc_encode_map(&set.maps1.m[3 + j], m->T[j], m->kpad_max, R, kTcBoxCols, kTcBoxRowsT);
        ok = ok && tc_encode_map(&set.maps2.m[3 + j], m->G[j], m->np_max, R, kTcBoxCols, kTcBoxRowsG);
    }
    for (int j = 0; j < 2; ++j)
        ok = ok && tc_encode_map(&set.maps1.m[6 + j], m->dT[j], m->kpad_max, R, kTcBoxCols, kTcBoxRowsT);
    if (!ok) {
        set_error_msg("gmco_solve_multi: cannot encode operand maps");
        return GMCO_ECUDA;
    }
    std::vector<TcDoseProb> dp((size_t)n);
    std::vector<TcGradProb> gp((size_t)n);
    std::vector<StepDesc> sd((size_t)2 * n);
    std::vector<int32_t> bstart((size_t)n + 1, 0);
    std::vector<int32_t *> cntp((size_t)n);
    m->st.assign((size_t)n, SolverState{});
    m->Wc_p.assign((size_t)n, nullptr);
    set.max_items1 = 0;
    set.max_items2 = 0;
    int64_t woff = 0;
    int32_t blocks = 0;
    for (int p = 0; p < n; ++p) {
        gmco_problem *pr = m->probs[p];
        const DevProblem &pb = pr->pb;
        const int32_t cap = (int32_t)P[p];
        SolverState s = pr->s;
        s.P = cap;
        m->st[p] = s;
        float *Fpart = nullptr, *dFpart = nullptr, *gpart = nullptr;
        const int32_t npt = tc_n_ptiles(pb);
        CK(a.alloc(&Fpart, (size_t)npt * cap));
        CK(a.alloc(&dFpart, (size_t)npt * cap));
        const SplitPlan sp = tc_split_plan(pb, m->split_kb, m->grad_tile);
        CK(a.alloc(&gpart, (size_t)max_split_rows(sp, cap) * pb.nd_pad));
        float *Wc = m->Wc + woff;
        woff += (int64_t)cap * pb.n_struct;
        m->Wc_p[p] = Wc;
        __nv_bfloat16 *Gp[3] = {nullptr, nullptr, nullptr};
        for (int j = 0; j < nT; ++j) Gp[j] = m->G[j] + m->t_row[p] * m->np_max;
        dp[p] = tc_dose_prob(pb, s.cnt, Wc, Gp, nullptr, Fpart, dFpart, (int32_t)m->a_row[p],
                             (int32_t)m->t_row[p], cap, (int32_t)m->np_max);
        gp[p] = tc_grad_prob(pb, s.cnt, gpart, sp, (int32_t)m->at_row[p], (int32_t)m->t_row[p]);
        set.max_items1 += ceil_div(cap, 128) * npt;
        set.max_items2 += ceil_div(cap, grad_bn(pb.tc_terms, m->grad_tile)) * tc_n_dtiles(pb) * sp.max_split;
        for (int par = 0; par < 2; ++par) {
            StepDesc &d = sd[(size_t)par * n + p];
            d.s = s;
            StepArgs &ar = d.a;
            ar = StepArgs{};
            ar.Fpart = Fpart;
            ar.dFpart = dFpart;
            ar.gpart = gpart;
            ar.n_ptiles = npt;
            ar.cap = cap;
            ar.sp = sp;
            ar.rows_cur = s.cnt + par;
            ar.rows_next = s.cnt + (par ^ 1);
            ar.fmt = 1;
            for (int j = 0; j < nT; ++j) ar.Tb[j] = m->T[j] + m->t_row[p] * m->kpad_max;
            for (int j = 0; j < 2; ++j) ar.dTb[j] = m->dT[j] + m->t_row[p] * m->kpad_max;
            ar.nT = nT;
            ar.kpad = (int32_t)pb.kpad;
            ar.ldT = (int32_t)m->kpad_max;
            ar.Wc = Wc;
        }
        bstart[p] = blocks;
        blocks += (int32_t)ceil_div(cap, 8);
        cntp[p] = s.cnt;
    }
    bstart[n] = blocks;
    m->total_blocks = blocks;
    TcDoseProb *d_dose = nullptr;
    TcGradProb *d_grad = nullptr;
    CK(a.alloc(&d_dose, (size_t)n));
    CK(a.alloc(&d_grad, (size_t)n));
    CK(a.alloc(&m->d_step, (size_t)2 * n));
    CK(a.alloc(&m->d_block_start, (size_t)n + 1));
    CK(a.alloc(&m->d_cnt, (size_t)n));
    CK(a.alloc(&m->d_sum, 1));
    CK(cudaMemcpy(d_dose, dp.data(), dp.size() * sizeof(TcDoseProb), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_grad, gp.data(), gp.size() * sizeof(TcGradProb), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->d_step, sd.data(), sd.size() * sizeof(StepDesc), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->d_block_start, bstart.data(), bstart.size() * sizeof(int32_t),
                  cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->d_cnt, cntp.data(), cntp.size() * sizeof(int32_t *), cudaMemcpyHostToDevice));
    set.dose = d_dose;
    set.grad = d_grad;
    set.n = n;
    set.tc_terms = m->tc_terms;
    set.err = m->err;
    set.wait_ns = (int64_t)m->probs[0]->opt.wait_limit_us * 1000;
    m->caps = P;
    m->gens = gens;
    m->ws_split = m->split_kb;
    m->ws_tile = m->grad_tile;
    return GMCO_OK;
}

TcRows multi_rows(const gmco_multi *m, int p)
{
    TcRows r{};
    const int nT = std::max(m->tc_terms, 2);
    for (int j = 0; j < nT; ++j) r.T[j] = m->T[j] + m->t_row[p] * m->kpad_max;
    for (int j = 0; j < 2; ++j) r.dT[j] = m->dT[j] + m->t_row[p] * m->kpad_max;
    r.Wc = m->Wc_p[p];
    r.ld = (int32_t)m->kpad_max;
    r.kpad = (int32_t)m->probs[p]->pb.kpad;
    r.nT = nT;
    return r;
}

// Stages weights and start times, checks them, and puts every plan in INIT with its first
// evaluation rows prepared.
gmco_status multi_start(gmco_multi *m, const float *const *W, const float *const *t0,
                        int32_t max_iters)
{
    for (int p = 0; p < m->n; ++p) {
        gmco_problem *pr = m->probs[p];
        const DevProblem &pb = pr->pb;
        const int64_t P = m->caps[p];
        CK(cudaMemcpyAsync(pr->dW, W[p], (size_t)P * pb.n_struct * sizeof(float), cudaMemcpyDefault,
                           m->stream));
        const bool has_t0 = t0 && t0[p];
        if (has_t0)
            CK(cudaMemcpyAsync(pr->dT0, t0[p], (size_t)P * pb.n_dwell * sizeof(float),
                               cudaMemcpyDefault, m->stream));
        CK(cudaMemsetAsync(pr->d_flag, 0, sizeof(int32_t), m->stream));
        k_count_bad<<<(unsigned)std::min<int64_t>(ceil_div(P * pb.n_struct, 256), 1184), 256, 0,
                      m->stream>>>(pr->dW, P * pb.n_struct, 0, pr->d_flag);
        if (has_t0)
            k_count_bad<<<(unsigned)std::min<int64_t>(ceil_div(P * pb.n_dwell, 256), 1184), 256, 0,
                          m->stream>>>(pr->dT0, P * pb.n_dwell, 0, pr->d_flag);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(m->h_pinned + 2 + p, pr->d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost,
                           m->stream));
        m->launches += has_t0 ? 2 : 1;
    }
    CK(cudaStreamSynchronize(m->stream));
    for (int p = 0; p < m->n; ++p)
        if (m->h_pinned[2 + p]) {
            char buf[160];
            snprintf(buf, sizeof buf,
                     "gmco_solve_multi: patient %d has negative or non-finite weights or start times", p);
            set_error_msg(buf);
            return GMCO_EINVAL;
        }
    for (int p = 0; p < m->n; ++p) {
        gmco_problem *pr = m->probs[p];
        const SolverState &s = m->st[p];
        CK(launch_solver_init(s, pr->pb, pr->dW, (t0 && t0[p]) ? pr->dT0 : nullptr, max_iters,
                              m->stream));
        CK(launch_compact(s, 0, m->stream));
        CK(tc_launch_prep(s, multi_rows(m, p), s.P, false, m->stream));
        m->launches += 3;
    }
    return GMCO_OK;
}

// Graph of `steps` (even) steps of every patient: dose GEMM (which also clears the next
// step's counters), gradient GEMM, fused update.
gmco_status multi_graph(gmco_multi *m, int steps, double tol)
{
    if (m->gexec && m->gkey_caps == m->caps && m->gkey_split == m->split_kb && m->gkey_tile == m->grad_tile &&
        m->gkey_steps == steps && m->gkey_tol == tol)
        return GMCO_OK;
    multi_destroy_graph(m);
    const UpdateParams u{m->opt.c1, tol, m->opt.max_ls, m->opt.stop_window, m->opt.max_evals};
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
        int32_t nl = 0;
        e = tc_launch_gemms(m->set, k & 1, true, false, true, m->stream, &nl);
        if (e == cudaSuccess)
            e = launch_step_multi(m->d_step + (size_t)(k & 1) * m->n, m->d_block_start, m->n,
                                  m->total_blocks, m->max_nd_pad, u, m->stream);
    }
    cudaError_t ee = cudaStreamEndCapture(m->stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        set_error("multi-patient step capture", e);
        return GMCO_ECUDA;
    }
    CK(ee);
    cudaError_t ei = cudaGraphInstantiate(&m->gexec, g, 0);
    cudaGraphDestroy(g);
    CK(ei);
    m->gkey_caps = m->caps;
    m->gkey_split = m->split_kb;
    m->gkey_tile = m->grad_tile;
    m->gkey_steps = steps;
    m->gkey_tol = tol;
    return GMCO_OK;
}

// Runs graphs until no patient has a plan left (or max_steps); counts launches.
gmco_status multi_loop(gmco_multi *m, int steps, int64_t max_steps, int64_t *done_out)
{
    int64_t done = 0;
    for (;;) {
        CK(cudaGraphLaunch(m->gexec, m->stream));
        m->launches += (int64_t)steps * 3;
        done += steps;
        CK(launch_sum_counters(m->d_cnt, m->n, m->d_sum, m->stream));
        m->launches++;
        CK(cudaMemcpyAsync(m->h_pinned, m->d_sum, sizeof(int32_t), cudaMemcpyDeviceToHost,
                           m->stream));
        CK(cudaStreamSynchronize(m->stream));
        if (m->h_pinned[0] == 0) break;
        if (done >= max_steps) {
            *done_out = done;
            return GMCO_ETIMEOUT;
        }
    }
    *done_out = done;
    return GMCO_OK;
}

gmco_status multi_check_err(gmco_multi *m)
{
    CK(cudaMemcpyAsync(m->h_pinned + 1, m->err, sizeof(int32_t), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    if (m->h_pinned[1] != 0) {
        char buf[128];
        snprintf(buf, sizeof buf, "tensor-core pipeline wait timed out (code %d)", m->h_pinned[1]);
        set_error_msg(buf);
        cudaMemsetAsync(m->err, 0, sizeof(int32_t), m->stream);
        return GMCO_ECUDA;
    }
    return GMCO_OK;
}

gmco_status multi_args(gmco_multi *m, const float *const *W, const int64_t *P,
                       std::vector<int64_t> *Pv, const char *who)
{
    if (!m || !W || !P) {
        set_error_msg((std::string(who) + ": null argument").c_str());
        return GMCO_EINVAL;
    }
    Pv->assign((size_t)m->n, 0);
    for (int p = 0; p < m->n; ++p) {
        if (!W[p] || P[p] < 1 || P[p] > (1 << 20)) {
            set_error_msg((std::string(who) + ": bad weights pointer or plan count").c_str());
            return GMCO_EINVAL;
        }
        (*Pv)[p] = P[p];
    }
    return GMCO_OK;
}

}  // namespace

extern "C" {

namespace {

// Device view of a caller buffer: the buffer itself when it is device memory, else a stream-
// ordered device copy (copied in when `in`); `back` copies a device copy out to the caller.
struct Staged {
    void *user = nullptr, *dev = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    bool own = false;
    ~Staged() { if (own && dev) cudaFreeAsync(dev, st); }
    cudaError_t init(void *p, size_t n, cudaStream_t s, bool in)
    {
        user = p;
        bytes = n;
        st = s;
        cudaPointerAttributes a{};
        bool on_dev = false;
        if (p && cudaPointerGetAttributes(&a, p) == cudaSuccess)
            on_dev = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
        cudaGetLastError();
        if (on_dev) {
            dev = p;
            return cudaSuccess;
        }
        own = true;
        cudaError_t e = cudaMallocAsync(&dev, n, s);
        if (e != cudaSuccess || !in || !p) return e;
        return cudaMemcpyAsync(dev, p, n, cudaMemcpyHostToDevice, s);
    }
    cudaError_t back() const
    {
        return (own && user) ? cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, st) : cudaSuccess;
    }
};

bool have_device()
{
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return false;
    }
    return true;
}

}  // namespace

void gmco_default_source(gmco_source *src)
{
    if (!src) return;
    src->lambda = 1.109;
    src->sk = 40700.0;
    src->unit = 1.0 / 360000.0;
    src->r_min = 0.1;
    src->g0 = 1.0;
    src->g1 = 0.005;
    src->g2 = -0.002;
}

gmco_status gmco_dose_rate_matrix(const float *points, int64_t n_pnt, const float *dwells,
                                  int64_t n_dwell, const gmco_source *src, float *A_out,
                                  void *cuda_stream)
{
    gmco_source m;
    gmco_default_source(&m);
    if (src) m = *src;
    const double c[7] = {m.lambda, m.sk, m.unit, m.r_min, m.g0, m.g1, m.g2};
    bool fin = true;
    for (double v : c) fin = fin && isfinite(v);
    if (!points || !dwells || !A_out || n_pnt < 1 || n_pnt > (1LL << 31) || n_dwell < 1 ||
        n_dwell > kMaxDwell || !fin || !(m.r_min > 0.0)) {
        set_error_msg("gmco_dose_rate_matrix: bad arguments");
        return GMCO_EINVAL;
    }
    if (!have_device()) {
        set_error_msg("gmco_dose_rate_matrix: no CUDA device");
        return GMCO_ECUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t pb = (size_t)n_pnt * 3 * sizeof(float), db = (size_t)n_dwell * 3 * sizeof(float);
    const size_t ab = (size_t)n_pnt * (size_t)n_dwell * sizeof(float);
    Staged P, D, Aw, flag;
    CK(P.init(const_cast<float *>(points), pb, st, true));
    CK(D.init(const_cast<float *>(dwells), db, st, true));
    CK(Aw.init(A_out, ab, st, false));
    CK(flag.init(nullptr, sizeof(int32_t), st, false));
    // non-finite coordinates give non-finite rates, caught with g(r) <= 0 by the kernel
    CK(cudaMemsetAsync(flag.dev, 0, sizeof(int32_t), st));
    CK(launch_dose_rate(static_cast<const float *>(P.dev), n_pnt, static_cast<const float *>(D.dev),
                        (int32_t)n_dwell, c, static_cast<float *>(Aw.dev), static_cast<int32_t *>(flag.dev), st));
    int32_t bad = 0;
    CK(cudaMemcpyAsync(&bad, flag.dev, sizeof bad, cudaMemcpyDeviceToHost, st));
    CK(Aw.back());
    CK(cudaStreamSynchronize(st));
    if (bad) {
        set_error_msg("gmco_dose_rate_matrix: g(r) <= 0 or a non-finite rate");
        return GMCO_EINVAL;
    }
    return GMCO_OK;
}


void gmco_default_rtog(gmco_rtog *c)
{
    if (!c) return;
    c->v100_min = 90.0;
    c->v100_min_plus = 95.0;
    c->d10_max = 118.0;
    c->v75_max_cc = 1.0;
    c->vol_cc[0] = c->vol_cc[1] = 0.0;
}

gmco_status gmco_rtog_select(const float *dvh, int64_t P, const gmco_rtog *crit, int32_t *cls,
                             int32_t *selected, void *cuda_stream)
{
    if (!dvh || !crit || !selected || P < 1 || P > (1LL << 30)) {
        set_error_msg("gmco_rtog_select: bad arguments");
        return GMCO_EINVAL;
    }
    const double c[6] = {crit->v100_min, crit->v100_min_plus, crit->d10_max, crit->v75_max_cc,
                         crit->vol_cc[0], crit->vol_cc[1]};
    for (double v : c)
        if (!isfinite(v)) {
            set_error_msg("gmco_rtog_select: non-finite criteria");
            return GMCO_EINVAL;
        }
    if (c[4] < 0.0 || c[5] < 0.0) {
        set_error_msg("gmco_rtog_select: negative volume");
        return GMCO_EINVAL;
    }
    if (!have_device()) {
        set_error_msg("gmco_rtog_select: no CUDA device");
        return GMCO_ECUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    Staged d, k, sc, ss;
    CK(d.init(const_cast<float *>(dvh), (size_t)P * GMCO_DVH_K * sizeof(float), st, true));
    CK(k.init(nullptr, sizeof c, st, false));
    CK(cudaMemcpyAsync(k.dev, c, sizeof c, cudaMemcpyHostToDevice, st));
    CK(sc.init(cls, (size_t)P * sizeof(int32_t), st, false));
    CK(ss.init(selected, sizeof(int32_t), st, false));
    CK(launch_rtog(static_cast<const float *>(d.dev), P, static_cast<const double *>(k.dev),
                   static_cast<int32_t *>(sc.dev), static_cast<int32_t *>(ss.dev), st));
    CK(sc.back());
    CK(ss.back());
    CK(cudaStreamSynchronize(st));
    return GMCO_OK;
}

gmco_status gmco_pareto_filter(const double *obj, int64_t P, int32_t K, int32_t *nondominated,
                               void *cuda_stream)
{
    if (!obj || !nondominated || P < 1 || P > (1LL << 30) || K < 1 || K > 16) {
        set_error_msg("gmco_pareto_filter: bad arguments");
        return GMCO_EINVAL;
    }
    if (!have_device()) {
        set_error_msg("gmco_pareto_filter: no CUDA device");
        return GMCO_ECUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    Staged o, n;
    CK(o.init(const_cast<double *>(obj), (size_t)P * K * sizeof(double), st, true));
    CK(n.init(nondominated, (size_t)P * sizeof(int32_t), st, false));
    CK(launch_pareto(static_cast<const double *>(o.dev), P, K, static_cast<int32_t *>(n.dev), st));
    CK(n.back());
    CK(cudaStreamSynchronize(st));
    return GMCO_OK;
}

void gmco_default_options(gmco_options *opt)
{
    if (!opt) return;
    opt->precision = GMCO_PREC_FP32;
    opt->m = 10;
    opt->c1 = 1e-4;
    opt->max_ls = 30;
    opt->rx_gy = 15.0;
    opt->refine_iters = 0;
    opt->steps_per_poll = 16;
    opt->stop_window = 1;
    opt->max_evals = 0;
    opt->grad_plan_tile = 0;
    opt->grad_split_kb = 0;
    opt->sparse_grad_permille = 0;
    opt->wait_limit_us = 1000000;
}

const char *gmco_status_string(gmco_status s)
{
    switch (s) {
    case GMCO_OK: return "ok";
    case GMCO_EINVAL: return "invalid argument";
    case GMCO_ENOMEM: return "device out of memory";
    case GMCO_ECUDA: return "CUDA error";
    case GMCO_ETIMEOUT: return "step budget exhausted with plans still running";
    case GMCO_EUNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

const char *gmco_last_error(void) { return g_last_error.c_str(); }

gmco_status gmco_create_problem(const float *A, int64_t n_pnt, int64_t n_dwell,
                                const int32_t *structure_ids, int32_t n_struct,
                                const double *penalty_params, const gmco_options *opt,
                                gmco_problem **out)
{
    if (!out) return GMCO_EINVAL;
    *out = nullptr;
    if (!A || !structure_ids || !penalty_params || n_pnt < 1 || n_dwell < 1 ||
        n_dwell > kMaxDwell || n_struct < 1 || n_struct > kMaxStruct || n_pnt > (1LL << 31)) {
        set_error_msg("gmco_create_problem: bad sizes or null pointer");
        return GMCO_EINVAL;
    }
    gmco_options o;
    gmco_default_options(&o);
    if (opt) o = *opt;
    if (o.precision < 0 || o.precision > 4 || o.m < 1 || o.m > kMaxHist || !(o.c1 > 0.0) ||
        !(o.c1 < 1.0) || o.max_ls < 1 || o.max_ls > 60 || !(o.rx_gy > 0.0) ||
        !isfinite(o.rx_gy) || o.refine_iters < 0 || o.steps_per_poll < 1 ||
        o.steps_per_poll > 1024 || o.stop_window < 1 || o.grad_split_kb < 0 || o.max_evals < 0 ||
        (o.grad_plan_tile != 0 && o.grad_plan_tile != 128 && o.grad_plan_tile != 256) ||
        o.sparse_grad_permille < 0 || o.sparse_grad_permille > 1000 || o.wait_limit_us < 1 ||
        o.wait_limit_us > 60000000) {
        set_error_msg("gmco_create_problem: bad options");
        return GMCO_EINVAL;
    }
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
        cudaGetLastError();
        set_error_msg("gmco_create_problem: no CUDA device");
        return GMCO_ECUDA;
    }
    // small host copies for validation (inputs may be host or device memory)
    std::vector<double> prm((size_t)n_struct * 4);
    std::vector<int32_t> sid((size_t)n_pnt);
    if (cudaMemcpy(prm.data(), penalty_params, prm.size() * sizeof(double), cudaMemcpyDefault) !=
            cudaSuccess ||
        cudaMemcpy(sid.data(), structure_ids, sid.size() * sizeof(int32_t), cudaMemcpyDefault) !=
            cudaSuccess) {
        set_error_msg("gmco_create_problem: cannot read structure ids / penalty params");
        cudaGetLastError();
        return GMCO_EINVAL;
    }
    std::vector<int64_t> counts((size_t)n_struct, 0);
    for (int64_t i = 0; i < n_pnt; ++i) {
        if (sid[i] < 0 || sid[i] >= n_struct) {
            set_error_msg("gmco_create_problem: structure id out of range");
            return GMCO_EINVAL;
        }
        counts[sid[i]]++;
    }
    for (int32_t s = 0; s < n_struct; ++s) {
        const double wmin = prm[4 * s], dmin = prm[4 * s + 1], dmax = prm[4 * s + 2],
                     wmax = prm[4 * s + 3];
        if (counts[s] == 0 || !isfinite(wmin) || !isfinite(wmax) || wmin < 0 || wmax < 0 ||
            isnan(dmin) || isnan(dmax) || dmin > dmax || dmin == INFINITY || dmax == -INFINITY) {
            set_error_msg("gmco_create_problem: empty structure or bad penalty parameters");
            return GMCO_EINVAL;
        }
    }

    gmco_problem *pr = new gmco_problem();
    pr->opt = o;
    pr->counts = counts;
    cudaGetDevice(&pr->device);
    auto fail = [&](gmco_status st) {
        gmco_destroy_problem(pr);
        return st;
    };
    auto ck = [&](cudaError_t e, const char *what) -> bool {
        if (e != cudaSuccess) {
            set_error(what, e);
            return false;
        }
        return true;
    };
    if (!ck(cudaStreamCreateWithFlags(&pr->stream, cudaStreamNonBlocking), "stream") ||
        !ck(cudaEventCreateWithFlags(&pr->ev_in, cudaEventDisableTiming), "event") ||
        !ck(cudaEventCreateWithFlags(&pr->ev_out, cudaEventDisableTiming), "event") ||
        !ck(cudaMallocHost(&pr->h_pinned, 64), "pinned") ||
        !ck(pr->arena.alloc(&pr->d_flag, 4), "flag"))
        return fail(GMCO_ECUDA);

    DevProblem &pb = pr->pb;
    pb.n_pnt = n_pnt;
    pb.n_dwell = n_dwell;
    pb.np_pad = round_up(n_pnt, 256);
    pb.nd_pad = round_up(n_dwell, 32);
    pb.n_struct = n_struct;
    const size_t an = (size_t)pb.np_pad * pb.nd_pad;
    if (!ck(pr->arena.alloc(&pb.A32, an), "alloc A") ||
        !ck(pr->arena.alloc(&pb.sid, (size_t)pb.np_pad), "alloc sid") ||
        !ck(pr->arena.alloc(&pb.sparams, (size_t)n_struct), "alloc params") ||
        !ck(pr->arena.alloc(&pb.inv_count, (size_t)n_struct), "alloc counts") ||
        !ck(pr->arena.alloc(&pb.row_scale, (size_t)pb.np_pad), "alloc scale"))
        return fail(GMCO_ENOMEM);
    if (!ck(cudaMemsetAsync(pb.A32, 0, an * sizeof(float), pr->stream), "memset A") ||
        !ck(cudaMemcpy2DAsync(pb.A32, pb.nd_pad * sizeof(float), A, n_dwell * sizeof(float),
                              n_dwell * sizeof(float), n_pnt, cudaMemcpyDefault, pr->stream),
            "copy A"))
        return fail(GMCO_ECUDA);
    int32_t bad = 0;
    if (count_bad(pr, pb.A32, (int64_t)an, false, &bad) != GMCO_OK) return fail(GMCO_ECUDA);
    if (bad) {
        set_error_msg("gmco_create_problem: A has negative or non-finite entries");
        return fail(GMCO_EINVAL);
    }
    std::vector<int8_t> sid8((size_t)pb.np_pad, (int8_t)-1);
    for (int64_t i = 0; i < n_pnt; ++i) sid8[i] = (int8_t)sid[i];
    std::vector<float4> sp((size_t)n_struct);
    std::vector<float> ic((size_t)n_struct);
    for (int32_t s = 0; s < n_struct; ++s) {
        sp[s] = make_float4((float)prm[4 * s], (float)prm[4 * s + 1], (float)prm[4 * s + 2],
                            (float)prm[4 * s + 3]);
        ic[s] = (float)(1.0 / (double)counts[s]);
    }
    if (!ck(cudaMemcpy(pb.sid, sid8.data(), sid8.size(), cudaMemcpyHostToDevice), "sid") ||
        !ck(cudaMemcpy(pb.sparams, sp.data(), sp.size() * sizeof(float4), cudaMemcpyHostToDevice),
            "params") ||
        !ck(cudaMemcpy(pb.inv_count, ic.data(), ic.size() * sizeof(float), cudaMemcpyHostToDevice),
            "counts"))
        return fail(GMCO_ECUDA);
    if (o.precision != GMCO_PREC_FP32) {
        cudaError_t e = tc_prepare_problem(&pb, o.precision, pr->stream,
                                           [&](void **p, size_t bytes) {
                                               unsigned char *q = nullptr;
                                               cudaError_t r = pr->arena.alloc(&q, bytes);
                                               *p = q;
                                               return r;
                                           });
        if (e == cudaErrorNotSupported) {
            set_error_msg("gmco_create_problem: tensor-core forms need n_dwell <= 512, n_struct <= 8");
            return fail(GMCO_EUNSUPPORTED);
        }
        if (!ck(e, "tensor-core problem setup")) return fail(GMCO_ECUDA);
    }
    if (!ck(cudaStreamSynchronize(pr->stream), "sync")) return fail(GMCO_ECUDA);
    *out = pr;
    return GMCO_OK;
}

void gmco_destroy_problem(gmco_problem *pr)
{
    if (!pr) return;
    cudaSetDevice(pr->device);
    if (pr->stream) cudaStreamSynchronize(pr->stream);
    destroy_graphs(pr);
    pr->ws_arena.release();
    pr->arena.release();
    if (pr->h_pinned) cudaFreeHost(pr->h_pinned);
    if (pr->ev_in) cudaEventDestroy(pr->ev_in);
    if (pr->ev_out) cudaEventDestroy(pr->ev_out);
    if (pr->stream) cudaStreamDestroy(pr->stream);
    delete pr;
}

gmco_status gmco_problem_info(const gmco_problem *pr, int64_t *n_pnt, int64_t *n_dwell,
                              int32_t *n_struct, int32_t *precision)
{
    if (!pr) return GMCO_EINVAL;
    if (n_pnt) *n_pnt = pr->pb.n_pnt;
    if (n_dwell) *n_dwell = pr->pb.n_dwell;
    if (n_struct) *n_struct = pr->pb.n_struct;
    if (precision) *precision = pr->opt.precision;
    return GMCO_OK;
}

int64_t gmco_last_launch_count(const gmco_problem *pr) { return pr ? pr->launches : -1; }

int64_t gmco_last_sparse_steps(const gmco_problem *pr)
{
    if (!pr || !pr->tcb.act) return -1;
    int32_t v = 0;
    if (cudaMemcpy(&v, pr->tcb.act + 4, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return v;
}

gmco_status gmco_solve_batch(gmco_problem *pr, const float *penalty_weights, int64_t P,
                             const float *t0, int32_t max_iters, double tol, float *T_out,
                             double *objectives, float *dvh, int32_t *iters_out,
                             int32_t *plan_status, void *cuda_stream)
{
    if (!pr || !penalty_weights || P < 1 || P > (1 << 20) || max_iters < 0 || !(tol >= 0.0) ||
        !isfinite(tol)) {
        set_error_msg("gmco_solve_batch: bad arguments");
        return GMCO_EINVAL;
    }
    pr->launches = 0;
    CKS(begin_call(pr, cuda_stream));
    CKS(ensure_workspace(pr, (int32_t)P));
    const DevProblem &pb = pr->pb;
    const int32_t S = pb.n_struct;
    CKS(stage_in(pr, penalty_weights, pr->dW, (size_t)P * S * sizeof(float)));
    if (t0) CKS(stage_in(pr, t0, pr->dT0, (size_t)P * pb.n_dwell * sizeof(float)));
    int32_t bad = 0;
    CKS(count_bad(pr, pr->dW, P * S, false, &bad));
    if (!bad && t0) {
        int32_t b2 = 0;
        CKS(count_bad(pr, pr->dT0, P * pb.n_dwell, false, &b2));
        bad += b2;
    }
    if (bad) {
        set_error_msg("gmco_solve_batch: negative or non-finite weights or start times");
        return GMCO_EINVAL;
    }
    // the plan-indexed state is sized for P plans in this call
    SolverState s = pr->s;
    s.P = (int32_t)P;
    SolverState saved = pr->s;
    pr->s = s;
    struct Restore {
        gmco_problem *p;
        SolverState st;
        ~Restore() { p->s = st; }
    } restore{pr, saved};

    CK(launch_solver_init(s, pb, pr->dW, t0 ? pr->dT0 : nullptr, max_iters, pr->stream));
    pr->launches++;
    UpdateParams u{pr->opt.c1, tol, pr->opt.max_ls, pr->opt.stop_window, pr->opt.max_evals};
    const int form = pr->opt.precision == GMCO_PREC_FP32 ? 0 : 1;
    const int64_t budget = ((int64_t)max_iters + pr->opt.refine_iters + 1) * (pr->opt.max_ls + 1) + 4;
    int64_t steps = 0;
    gmco_status rs = run_loop(pr, form, (int32_t)P, u, budget, &steps);
    if (rs != GMCO_OK && rs != GMCO_ETIMEOUT) return rs;
    if (rs == GMCO_OK && form != 0 && pr->opt.refine_iters > 0) {
        CK(launch_reopen(s, pr->opt.refine_iters, pr->stream));
        pr->launches++;
        int64_t steps2 = 0;
        rs = run_loop(pr, 0, (int32_t)P, u, budget, &steps2);
        if (rs != GMCO_OK && rs != GMCO_ETIMEOUT) return rs;
    }
    CKS(check_tc_error(pr));
    // final FP32 evaluation at x: objectives and doses (for the DVH indices)
    CKS(launch_dose_eval(pr, s, pr->stream));
    if (dvh) {
        CK(launch_dvh(pb, pr->G, pb.np_pad, s.list, (int32_t)P, pr->opt.rx_gy, pr->dDvh,
                      pr->stream));
        pr->launches++;
        CK(cudaMemcpyAsync(dvh, pr->dDvh, (size_t)P * GMCO_DVH_K * sizeof(float),
                           cudaMemcpyDefault, pr->stream));
    }
    if (T_out) {
        CK(launch_square(s.x, pr->dTout, P, pb.n_dwell, pb.nd_pad, pr->stream));
        pr->launches++;
        CK(cudaMemcpyAsync(T_out, pr->dTout, (size_t)P * pb.n_dwell * sizeof(float),
                           cudaMemcpyDefault, pr->stream));
    }
    if (objectives)
        CK(cudaMemcpyAsync(objectives, s.Ft, (size_t)P * sizeof(double), cudaMemcpyDefault,
                           pr->stream));
    if (iters_out)
        CK(cudaMemcpyAsync(iters_out, s.iters, (size_t)P * sizeof(int32_t), cudaMemcpyDefault,
                           pr->stream));
    if (plan_status)
        CK(cudaMemcpyAsync(plan_status, s.status, (size_t)P * sizeof(int32_t),
                           cudaMemcpyDefault, pr->stream));
    CKS(end_call(pr, cuda_stream));
    return rs;
}

gmco_status gmco_evaluate(gmco_problem *pr, const float *penalty_weights, int64_t P,
                          const float *X, double *objectives, float *grad_x, float *dose,
                          float *dvh, void *cuda_stream)
{
    if (!pr || !penalty_weights || !X || P < 1 || P > (1 << 20)) {
        set_error_msg("gmco_evaluate: bad arguments");
        return GMCO_EINVAL;
    }
    pr->launches = 0;
    CKS(begin_call(pr, cuda_stream));
    CKS(ensure_workspace(pr, (int32_t)P));
    const DevProblem &pb = pr->pb;
    const int32_t S = pb.n_struct;
    CKS(stage_in(pr, penalty_weights, pr->dW, (size_t)P * S * sizeof(float)));
    CKS(stage_in(pr, X, pr->dT0, (size_t)P * pb.n_dwell * sizeof(float)));
    int32_t bad = 0, b2 = 0;
    CKS(count_bad(pr, pr->dW, P * S, false, &bad));
    CKS(count_bad(pr, pr->dT0, P * pb.n_dwell, true, &b2));
    if (bad || b2) {
        set_error_msg("gmco_evaluate: negative weights or non-finite inputs");
        return GMCO_EINVAL;
    }
    SolverState s = pr->s;
    s.P = (int32_t)P;
    SolverState saved = pr->s;
    pr->s = s;
    struct Restore {
        gmco_problem *p;
        SolverState st;
        ~Restore() { p->s = st; }
    } restore{pr, saved};
    CK(launch_solver_init(s, pb, pr->dW, nullptr, 0, pr->stream));
    CK(cudaMemcpy2DAsync(s.x, pb.nd_pad * sizeof(float), pr->dT0, pb.n_dwell * sizeof(float),
                         pb.n_dwell * sizeof(float), P, cudaMemcpyDeviceToDevice, pr->stream));
    pr->launches++;
    const int form = pr->opt.precision == GMCO_PREC_FP32 ? 0 : 1;
    if (objectives || grad_x) {
        CK(launch_compact(s, 0, pr->stream));
        pr->launches++;
        CKS(launch_eval(pr, s, form, false, pr->stream));
        if (objectives)
            CK(cudaMemcpyAsync(objectives, s.Ft, (size_t)P * sizeof(double), cudaMemcpyDefault,
                               pr->stream));
        if (grad_x)
            CK(cudaMemcpy2DAsync(grad_x, pb.n_dwell * sizeof(float), s.gt,
                                 pb.nd_pad * sizeof(float), pb.n_dwell * sizeof(float), P,
                                 cudaMemcpyDefault, pr->stream));
    }
    if (dose || dvh) {
        if (form == 0) {
            CKS(launch_dose_eval(pr, s, pr->stream));
        } else {
            CK(launch_compact(s, 1, pr->stream));
            int32_t nl = 0;
            CK(tc_launch_eval(pb, s, pr->tcb, pr->cap, false, true, true, pr->stream, &nl));
            pr->launches += nl + 1;
        }
        if (dose)
            CK(cudaMemcpy2DAsync(dose, pb.n_pnt * sizeof(float), pr->G, pb.np_pad * sizeof(float),
                                 pb.n_pnt * sizeof(float), P, cudaMemcpyDefault, pr->stream));
        if (dvh) {
            CK(launch_dvh(pb, pr->G, pb.np_pad, s.list, (int32_t)P, pr->opt.rx_gy, pr->dDvh,
                          pr->stream));
            pr->launches++;
            CK(cudaMemcpyAsync(dvh, pr->dDvh, (size_t)P * GMCO_DVH_K * sizeof(float),
                               cudaMemcpyDefault, pr->stream));
        }
    }
    CKS(check_tc_error(pr));
    CKS(end_call(pr, cuda_stream));
    return GMCO_OK;
}

void gmco_default_sa_options(gmco_sa_options *opt)
{
    if (!opt) return;
    opt->iterations = 1000;
    opt->seed = 1;
    opt->T0 = 1e-2;
    opt->T_final = 1e-5;
    opt->step0 = 0.2;
    opt->step_final = 2e-3;
}

namespace {

// Geometric interpolation from a to b over K iterations: a (b / a)^(k / (K - 1)); 0 when a = 0.
double sa_schedule(double a, double b, int32_t k, int32_t K)
{
    if (a == 0.0) return 0.0;
    const double f = K > 1 ? (double)k / (double)(K - 1) : 0.0;
    return a * pow(b / a, f);
}

bool sa_pair_ok(double a, double b)
{
    return isfinite(a) && isfinite(b) && a >= 0.0 && b >= 0.0 && ((a == 0.0) == (b == 0.0));
}

}  // namespace

gmco_status gmco_solve_sa(gmco_problem *pr, const float *penalty_weights, int64_t P,
                          const float *t0, const gmco_sa_options *opt, float *T_out,
                          double *objectives, int32_t *accepts, void *cuda_stream)
{
    if (!pr || !penalty_weights || !opt || P < 1 || P >= (1 << 21) || opt->iterations < 0 ||
        opt->iterations >= (1 << 22) || !sa_pair_ok(opt->T0, opt->T_final) ||
        !sa_pair_ok(opt->step0, opt->step_final) || pr->pb.n_dwell >= (1 << 21) - 1) {
        set_error_msg("gmco_solve_sa: bad arguments");
        return GMCO_EINVAL;
    }
    pr->launches = 0;
    CKS(begin_call(pr, cuda_stream));
    CKS(ensure_workspace(pr, (int32_t)P));
    const DevProblem &pb = pr->pb;
    const int32_t S = pb.n_struct;
    CKS(stage_in(pr, penalty_weights, pr->dW, (size_t)P * S * sizeof(float)));
    if (t0) CKS(stage_in(pr, t0, pr->dT0, (size_t)P * pb.n_dwell * sizeof(float)));
    int32_t bad = 0;
    CKS(count_bad(pr, pr->dW, P * S, false, &bad));
    if (!bad && t0) {
        int32_t b2 = 0;
        CKS(count_bad(pr, pr->dT0, P * pb.n_dwell, false, &b2));
        bad += b2;
    }
    if (bad) {
        set_error_msg("gmco_solve_sa: negative or non-finite weights or start times");
        return GMCO_EINVAL;
    }
    SolverState s = pr->s;
    s.P = (int32_t)P;
    SolverState saved = pr->s;
    pr->s = s;
    struct Restore {
        gmco_problem *p;
        SolverState st;
        ~Restore() { p->s = st; }
    } restore{pr, saved};
    cudaStream_t st = pr->stream;
    CK(launch_solver_init(s, pb, pr->dW, t0 ? pr->dT0 : nullptr, 0, st));
    pr->launches++;
    // The annealing keeps its state in the solver workspace: s.x holds the moved weights that
    // the evaluation reads, s.g the current and s.p the best weights; s.F, s.alpha and s.gtp the
    // current, best and start objectives; s.iters the accepted moves.
    float *xc = s.g, *xb = s.p;
    double *Fc = s.F, *Fb = s.alpha, *F0 = s.gtp;
    const int form = pr->opt.precision == GMCO_PREC_FP32 ? 0 : 1;
    if (form != 0) {
        CK(launch_compact(s, 1, st));   // every plan, every iteration
        pr->launches++;
    }
    auto evaluate_all = [&]() -> gmco_status {
        if (form == 0) return launch_dose_eval(pr, s, st);
        int32_t nl = 0;
        CK(tc_launch_eval(pb, s, pr->tcb, pr->cap, false, true, true, st, &nl));
        pr->launches += nl;
        return GMCO_OK;
    };
    const uint64_t seed = opt->seed;
    CKS(evaluate_all());
    CK(launch_sa_accept(s.x, xc, xb, P, pb.nd_pad, s.Ft, Fc, Fb, F0, s.iters, seed, -1, 0.0, st));
    pr->launches++;
    const int32_t K = opt->iterations;
    for (int32_t k = 0; k < K; ++k) {
        const double delta = sa_schedule(opt->step0, opt->step_final, k, K);
        const double temp = sa_schedule(opt->T0, opt->T_final, k, K);
        CK(launch_sa_propose(s.x, xc, P, pb.n_dwell, pb.nd_pad, seed, k, delta, st));
        CKS(evaluate_all());
        CK(launch_sa_accept(s.x, xc, xb, P, pb.nd_pad, s.Ft, Fc, Fb, F0, s.iters, seed, k, temp, st));
        pr->launches += 2;
    }
    CKS(check_tc_error(pr));
    if (T_out) {
        CK(launch_square(xb, pr->dTout, P, pb.n_dwell, pb.nd_pad, st));
        pr->launches++;
        CK(cudaMemcpyAsync(T_out, pr->dTout, (size_t)P * pb.n_dwell * sizeof(float),
                           cudaMemcpyDefault, st));
    }
    if (objectives)
        CK(cudaMemcpyAsync(objectives, Fb, (size_t)P * sizeof(double), cudaMemcpyDefault, st));
    if (accepts)
        CK(cudaMemcpyAsync(accepts, s.iters, (size_t)P * sizeof(int32_t), cudaMemcpyDefault, st));
    CKS(end_call(pr, cuda_stream));
    return GMCO_OK;
}

gmco_status gmco_profile_evaluate(gmco_problem *pr, const float *penalty_weights, int64_t P,
                                  const float *X, int32_t reps, double *ms, double *flops)
{
    if (!pr || !penalty_weights || !X || !ms || P < 1 || P > (1 << 20) || reps < 1 || reps > 1000) {
        set_error_msg("gmco_profile_evaluate: bad arguments");
        return GMCO_EINVAL;
    }
    pr->launches = 0;
    CKS(begin_call(pr, nullptr));
    CKS(ensure_workspace(pr, (int32_t)P));
    const DevProblem &pb = pr->pb;
    const int32_t S = pb.n_struct;
    CKS(stage_in(pr, penalty_weights, pr->dW, (size_t)P * S * sizeof(float)));
    CKS(stage_in(pr, X, pr->dT0, (size_t)P * pb.n_dwell * sizeof(float)));
    SolverState s = pr->s;
    s.P = (int32_t)P;
    SolverState saved = pr->s;
    pr->s = s;
    struct Restore {
        gmco_problem *p;
        SolverState st;
        ~Restore() { p->s = st; }
    } restore{pr, saved};
    CK(launch_solver_init(s, pb, pr->dW, nullptr, 0, pr->stream));
    CK(cudaMemcpy2DAsync(s.x, pb.nd_pad * sizeof(float), pr->dT0, pb.n_dwell * sizeof(float),
                         pb.n_dwell * sizeof(float), P, cudaMemcpyDeviceToDevice, pr->stream));
    CK(launch_profile_setup(s, pr->stream));
    CK(launch_compact(s, 0, pr->stream));
    const int form = pr->opt.precision == GMCO_PREC_FP32 ? 0 : 1;
    // the repetitions run back to back on the stream, as the solve loop's launches do (no
    // synchronisation between them, which would add an idle GPU's launch latency to each
    // kernel's time); one set of events per repetition, the first repetition a warm-up
    std::vector<cudaEvent_t> ev((size_t)5 * (reps + 1), nullptr);
    gmco_status rs = GMCO_OK;
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) rs = GMCO_ECUDA;
    for (int r = 0; r < reps + 1 && rs == GMCO_OK; ++r) rs = launch_eval(pr, s, form, true, pr->stream, &ev[(size_t)5 * r]);
    if (rs == GMCO_OK && cudaStreamSynchronize(pr->stream) != cudaSuccess) rs = GMCO_ECUDA;
    double acc[4] = {0, 0, 0, 0};
    for (int r = 1; r < reps + 1 && rs == GMCO_OK; ++r)
        for (int k = 0; k < 4; ++k) {
            float t = 0.0f;
            cudaEventElapsedTime(&t, ev[(size_t)5 * r + k], ev[(size_t)5 * r + k + 1]);
            acc[k] += t;
        }
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    if (rs != GMCO_OK) return rs;
    for (int k = 0; k < 4; ++k) ms[k] = acc[k] / reps;
    if (flops) {
        // algorithmic, the method's count: the dose d = A t of Eq. (dose) and the gradient
        // contraction A^T G of Eq. (2), one 2 P n_pnt n_dwell each.  The dose change dd that the
        // dose GEMM also forms for the line search is this library's numerical device, not
        // work of the method, and is left out (it is in the issued figure).
        const double c = 2.0 * (double)P * (double)pb.n_pnt * (double)pb.n_dwell;
        flops[0] = c;
        flops[1] = c;
        // issued on the tensor cores (split terms, padded tiles); FP32 form: algorithmic
        if (form == 1) {
            const double cp = 2.0 * (double)round_up(P, 128) * (double)pb.np_pad *
                              (double)round_up(pb.n_dwell, 16);
            flops[2] = tc_mma_units(pb, true, 1) * cp;
            flops[3] = tc_mma_units(pb, true, 2) * cp;
        } else {
            flops[2] = 2.0 * c;   // d and dd
            flops[3] = c;
        }
    }
    CKS(check_tc_error(pr));
    CKS(end_call(pr, nullptr));
    return GMCO_OK;
}

gmco_status gmco_evaluate_noalloc(const gmco_problem *pr, const float *penalty_weights,
                                  int64_t P, const float *X, double *objectives, float *grad_x,
                                  void *cuda_stream)
{
    if (!pr || !penalty_weights || !X || (!objectives && !grad_x) || P < 1 || P > (1 << 20)) {
        set_error_msg("gmco_evaluate_noalloc: bad arguments");
        return GMCO_EINVAL;
    }
    // every buffer must already be device memory: staging host data would need scratch
    const void *ptrs[4] = {penalty_weights, X, objectives, grad_x};
    for (const void *q : ptrs) {
        if (!q) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
            cudaGetLastError();
            set_error_msg("gmco_evaluate_noalloc: buffers must be device memory");
            return GMCO_EINVAL;
        }
        if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
            set_error_msg("gmco_evaluate_noalloc: buffers must be device memory");
            return GMCO_EINVAL;
        }
        if (a.type == cudaMemoryTypeDevice && a.device != pr->device) {
            set_error_msg("gmco_evaluate_noalloc: buffers must be on the problem's device");
            return GMCO_EINVAL;
        }
    }
    const size_t need = noalloc_required_bytes(pr->pb, P);
    if (need > noalloc_scratch_bytes()) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "gmco_evaluate_noalloc: %lld plans of this problem need %zu bytes of scratch; "
                 "the fixed scratch array holds %zu bytes",
                 (long long)P, need, noalloc_scratch_bytes());
        set_error_msg(buf);
        return GMCO_EUNSUPPORTED;
    }
    CK(cudaSetDevice(pr->device));
    CK(noalloc_evaluate(pr->pb, penalty_weights, P, X, objectives, grad_x,
                        (cudaStream_t)cuda_stream));
    return GMCO_OK;
}

gmco_status gmco_sample_points(const gmco_geometry *geo, const int64_t *counts, uint64_t seed,
                               float *points, int32_t *sid, void *cuda_stream)
{
    if (!geo || !counts || !points || !sid) {
        set_error_msg("gmco_sample_points: null pointer");
        return GMCO_EINVAL;
    }
    const double g[9] = {geo->a, geo->b, geo->c, geo->urethra_r, geo->rectum_r, geo->rectum_y,
                         geo->rectum_half_len, geo->bladder_r, geo->bladder_z};
    for (int i = 0; i < 9; ++i)
        if (!isfinite(g[i]) || (i != 5 && i != 8 && !(g[i] > 0.0))) {
            set_error_msg("gmco_sample_points: sizes must be finite and positive, centres finite");
            return GMCO_EINVAL;
        }
    int64_t total = 0;
    for (int s = 0; s < 4; ++s) {
        if (counts[s] < 0 || counts[s] > (1LL << 31)) {
            set_error_msg("gmco_sample_points: bad point count");
            return GMCO_EINVAL;
        }
        total += counts[s];
    }
    if (total < 1 || total > (1LL << 31)) {
        set_error_msg("gmco_sample_points: total point count outside 1..2^31");
        return GMCO_EINVAL;
    }
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
        cudaGetLastError();
        set_error_msg("gmco_sample_points: no CUDA device");
        return GMCO_ECUDA;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // outputs in host memory are written through device buffers
    auto on_device = [](const void *q) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    };
    const bool dp = on_device(points), ds = on_device(sid);
    float *d_pts = points;
    int32_t *d_sid = sid;
    if (!dp) CK(cudaMalloc(&d_pts, (size_t)total * 3 * sizeof(float)));
    if (!ds && cudaMalloc(&d_sid, (size_t)total * sizeof(int32_t)) != cudaSuccess) {
        if (!dp) cudaFree(d_pts);
        set_error_msg("gmco_sample_points: device allocation failed");
        return GMCO_ENOMEM;
    }
    int32_t short_s = -1;
    cudaError_t e = sample_points_dev(g, counts, seed, d_pts, d_sid, st, &short_s);
    if (e == cudaSuccess && !dp)
        e = cudaMemcpyAsync(points, d_pts, (size_t)total * 3 * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && !ds)
        e = cudaMemcpyAsync(sid, d_sid, (size_t)total * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (!dp) cudaFree(d_pts);
    if (!ds) cudaFree(d_sid);
    if (e != cudaSuccess) {
        set_error("gmco_sample_points", e);
        return GMCO_ECUDA;
    }
    if (short_s >= 0) {
        char buf[160];
        snprintf(buf, sizeof buf,
                 "gmco_sample_points: structure %d accepts too few candidates (empty or covered "
                 "by the structures it excludes)", short_s);
        set_error_msg(buf);
        return GMCO_EINVAL;
    }
    return GMCO_OK;
}

gmco_status gmco_dvh_at(gmco_problem *pr, const float *T, int64_t P, float *dvh, void *cuda_stream)
{
    if (!pr || !T || !dvh || P < 1 || P > (1 << 20)) {
        set_error_msg("gmco_dvh_at: bad arguments");
        return GMCO_EINVAL;
    }
    pr->launches = 0;
    CKS(begin_call(pr, cuda_stream));
    CKS(ensure_workspace(pr, (int32_t)P));
    const DevProblem &pb = pr->pb;
    CKS(stage_in(pr, T, pr->dT0, (size_t)P * pb.n_dwell * sizeof(float)));
    int32_t bad = 0;
    CKS(count_bad(pr, pr->dT0, P * pb.n_dwell, false, &bad));
    if (bad) {
        set_error_msg("gmco_dvh_at: negative or non-finite dwell times");
        return GMCO_EINVAL;
    }
    const SolverState &s = pr->s;
    k_rows_from_times<<<(unsigned)P, 128, 0, pr->stream>>>(pr->dT0, (int32_t)P, (int32_t)pb.n_dwell,
                                                          (int32_t)pb.nd_pad, pb.n_struct, pr->Tc,
                                                          pr->Wc, s.list, s.n_act);
    CK(cudaGetLastError());
    // the doses A t with the FP32 form, into the rows of G (dose mode)
    EvalArgs e{};
    e.pb = pb;
    e.n_rows = s.n_act;
    e.cap = pr->cap;
    e.Tt = pr->Tc;
    e.dT = nullptr;
    e.Wc = pr->Wc;
    e.G = pr->G;
    e.Fpart = pr->Fpart;
    e.dFpart = nullptr;
    e.gpart = nullptr;
    e.sp = simt_split_plan(pb);
    CK(launch_gemm1_simt(e, MODE_DOSE, pr->stream));
    CK(launch_dvh(pb, pr->G, pb.np_pad, s.list, (int32_t)P, pr->opt.rx_gy, pr->dDvh, pr->stream));
    pr->launches += 3;
    CK(cudaMemcpyAsync(dvh, pr->dDvh, (size_t)P * GMCO_DVH_K * sizeof(float), cudaMemcpyDefault,
                       pr->stream));
    CKS(end_call(pr, cuda_stream));
    return GMCO_OK;
}

gmco_status gmco_dvh_from_dose(gmco_problem *pr, const float *dose, int64_t P, float *dvh,
                               void *cuda_stream)
{
    if (!pr || !dose || !dvh || P < 1 || P > (1 << 20)) {
        set_error_msg("gmco_dvh_from_dose: bad arguments");
        return GMCO_EINVAL;
    }
    pr->launches = 0;
    CKS(begin_call(pr, cuda_stream));
    CKS(ensure_workspace(pr, (int32_t)P));
    const DevProblem &pb = pr->pb;
    const int64_t need = P * pb.n_pnt;
    if (need > pr->dose_cap) {
        CK(pr->ws_arena.alloc(&pr->dDose, (size_t)need));
        pr->dose_cap = need;
    }
    CKS(stage_in(pr, dose, pr->dDose, (size_t)need * sizeof(float)));
    int32_t bad = 0;
    CKS(count_bad(pr, pr->dDose, need, true, &bad));
    if (bad) {
        set_error_msg("gmco_dvh_from_dose: non-finite doses");
        return GMCO_EINVAL;
    }
    CK(launch_dvh(pb, pr->dDose, pb.n_pnt, nullptr, (int32_t)P, pr->opt.rx_gy, pr->dDvh,
                  pr->stream));
    pr->launches++;
    CK(cudaMemcpyAsync(dvh, pr->dDvh, (size_t)P * GMCO_DVH_K * sizeof(float), cudaMemcpyDefault,
                       pr->stream));
    CKS(end_call(pr, cuda_stream));
    return GMCO_OK;
}


gmco_status gmco_create_multi(gmco_problem *const *probs, int32_t n, gmco_multi **out)
{
    if (!out) return GMCO_EINVAL;
    *out = nullptr;
    if (!probs || n < 1 || n > kMaxMulti) {
        set_error_msg("gmco_create_multi: need 1..64 problems");
        return GMCO_EINVAL;
    }
    for (int p = 0; p < n; ++p) {
        if (!probs[p]) {
            set_error_msg("gmco_create_multi: null problem");
            return GMCO_EINVAL;
        }
        for (int q = 0; q < p; ++q)
            if (probs[q] == probs[p]) {
                set_error_msg("gmco_create_multi: a problem appears twice");
                return GMCO_EINVAL;
            }
    }
    const gmco_options &o = probs[0]->opt;
    for (int p = 0; p < n; ++p) {
        const gmco_problem *pr = probs[p];
        if (pr->opt.precision == GMCO_PREC_FP32) {
            set_error_msg("gmco_create_multi: the FP32 form has no multi-patient launch; use a "
                          "tensor-core precision");
            return GMCO_EUNSUPPORTED;
        }
        const gmco_options &q = pr->opt;
        if (q.precision != o.precision || q.m != o.m || q.c1 != o.c1 || q.max_ls != o.max_ls ||
            q.stop_window != o.stop_window || q.max_evals != o.max_evals ||
            q.grad_plan_tile != o.grad_plan_tile ||
            q.steps_per_poll != o.steps_per_poll || q.wait_limit_us != o.wait_limit_us ||
            pr->device != probs[0]->device) {
            set_error_msg("gmco_create_multi: problems differ in precision, solver options or device");
            return GMCO_EINVAL;
        }
    }
    gmco_multi *m = new gmco_multi();
    m->device = probs[0]->device;
    m->grad_tile = o.grad_plan_tile;
    m->probs.assign(probs, probs + n);
    m->n = n;
    m->opt = o;
    m->tc_terms = probs[0]->pb.tc_terms;
    auto fail = [&](gmco_status st) {
        gmco_destroy_multi(m);
        return st;
    };
    auto ck = [&](cudaError_t e, const char *what) -> bool {
        if (e != cudaSuccess) {
            set_error(what, e);
            return false;
        }
        return true;
    };
    if (!ck(cudaSetDevice(m->device), "device") ||
        !ck(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking), "stream") ||
        !ck(cudaEventCreateWithFlags(&m->ev_in, cudaEventDisableTiming), "event") ||
        !ck(cudaEventCreateWithFlags(&m->ev_out, cudaEventDisableTiming), "event") ||
        !ck(cudaMallocHost(&m->h_pinned, 256 * sizeof(int32_t)), "pinned") ||
        !ck(m->arena.alloc(&m->err, 1), "flag") || !ck(cudaMemset(m->err, 0, 4), "flag"))
        return fail(GMCO_ECUDA);
    m->a_row.assign((size_t)n, 0);
    m->at_row.assign((size_t)n, 0);
    for (int p = 0; p < n; ++p) {
        const DevProblem &pb = probs[p]->pb;
        m->a_row[p] = m->rows_A;
        m->at_row[p] = m->rows_AT;
        m->rows_A += pb.np_pad;
        m->rows_AT += pb.kpad;
        m->kpad_max = std::max(m->kpad_max, pb.kpad);
        m->np_max = std::max(m->np_max, pb.np_pad);
        m->max_nd_pad = std::max(m->max_nd_pad, (int32_t)pb.nd_pad);
    }
    for (int i = 0; i < m->tc_terms; ++i) {
        const size_t na = (size_t)m->rows_A * m->kpad_max, nat = (size_t)m->rows_AT * m->np_max;
        if (!ck(m->arena.alloc(&m->Ah[i], na), "alloc stacked A") ||
            !ck(m->arena.alloc(&m->AhT[i], nat), "alloc stacked A^T"))
            return fail(GMCO_ENOMEM);
        if (!ck(cudaMemsetAsync(m->Ah[i], 0, na * 2, m->stream), "memset") ||
            !ck(cudaMemsetAsync(m->AhT[i], 0, nat * 2, m->stream), "memset"))
            return fail(GMCO_ECUDA);
        for (int p = 0; p < n; ++p) {
            const DevProblem &pb = probs[p]->pb;
            if (!ck(cudaMemcpy2DAsync(m->Ah[i] + m->a_row[p] * m->kpad_max, m->kpad_max * 2, pb.Ah[i],
                                      pb.kpad * 2, pb.kpad * 2, pb.np_pad, cudaMemcpyDeviceToDevice,
                                      m->stream),
                    "stack A") ||
                !ck(cudaMemcpy2DAsync(m->AhT[i] + m->at_row[p] * m->np_max, m->np_max * 2, pb.AhT[i],
                                      pb.np_pad * 2, pb.np_pad * 2, pb.kpad, cudaMemcpyDeviceToDevice,
                                      m->stream),
                    "stack A^T"))
                return fail(GMCO_ECUDA);
        }
    }
    if (!ck(cudaStreamSynchronize(m->stream), "sync")) return fail(GMCO_ECUDA);
    *out = m;
    return GMCO_OK;
}

void gmco_destroy_multi(gmco_multi *m)
{
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    multi_destroy_graph(m);
    m->ws.release();
    m->arena.release();
    if (m->h_pinned) cudaFreeHost(m->h_pinned);
    if (m->ev_in) cudaEventDestroy(m->ev_in);
    if (m->ev_out) cudaEventDestroy(m->ev_out);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

gmco_status gmco_multi_set_split(gmco_multi *m, int32_t split_kb)
{
    if (!m || split_kb < 0) {
        set_error_msg("gmco_multi_set_split: bad arguments");
        return GMCO_EINVAL;
    }
    m->split_kb = split_kb;
    return GMCO_OK;
}

int32_t gmco_multi_get_split(const gmco_multi *m) { return m ? m->split_kb : -1; }

gmco_status gmco_multi_set_tiles(gmco_multi *m, int32_t split_kb, int32_t grad_plan_tile)
{
    if (!m || split_kb < 0 || (grad_plan_tile != 0 && grad_plan_tile != 128 && grad_plan_tile != 256)) {
        set_error_msg("gmco_multi_set_tiles: bad arguments");
        return GMCO_EINVAL;
    }
    m->split_kb = split_kb;
    m->grad_tile = grad_plan_tile;
    return GMCO_OK;
}

int32_t gmco_multi_get_grad_tile(const gmco_multi *m) { return m ? m->grad_tile : -1; }

int64_t gmco_multi_last_launch_count(const gmco_multi *m) { return m ? m->launches : -1; }

gmco_status gmco_solve_multi(gmco_multi *m, const float *const *penalty_weights,
                             const int64_t *P, const float *const *t0, int32_t max_iters,
                             double tol, float *const *T_out, double *const *objectives,
                             float *const *dvh, int32_t *const *iters_out,
                             int32_t *const *plan_status, void *cuda_stream)
{
    std::vector<int64_t> Pv;
    CKS(multi_args(m, penalty_weights, P, &Pv, "gmco_solve_multi"));
    if (max_iters < 0 || !(tol >= 0.0) || !isfinite(tol)) {
        set_error_msg("gmco_solve_multi: bad arguments");
        return GMCO_EINVAL;
    }
    m->launches = 0;
    CK(cudaSetDevice(m->device));
    CK(cudaEventRecord(m->ev_in, (cudaStream_t)cuda_stream));
    CK(cudaStreamWaitEvent(m->stream, m->ev_in, 0));
    CKS(multi_workspace(m, Pv));
    CKS(multi_start(m, penalty_weights, t0, max_iters));
    const int steps = (int)round_up(std::max(2, m->opt.steps_per_poll), 2);
    CKS(multi_graph(m, steps, tol));
    const int64_t budget = ((int64_t)max_iters + 1) * (m->opt.max_ls + 1) + 4;
    int64_t done = 0;
    gmco_status rs = multi_loop(m, steps, budget, &done);
    if (rs != GMCO_OK && rs != GMCO_ETIMEOUT) return rs;
    CKS(multi_check_err(m));
    for (int p = 0; p < m->n; ++p) {
        gmco_problem *pr = m->probs[p];
        const DevProblem &pb = pr->pb;
        const SolverState &s = m->st[p];
        const int64_t Pp = Pv[p];
        // final FP32 evaluation at x: objectives and doses (for the DVH indices)
        CKS(launch_dose_eval(pr, s, m->stream));
        m->launches += 4;
        if (dvh && dvh[p]) {
            CK(launch_dvh(pb, pr->G, pb.np_pad, s.list, (int32_t)Pp, m->opt.rx_gy, pr->dDvh,
                          m->stream));
            m->launches++;
            CK(cudaMemcpyAsync(dvh[p], pr->dDvh, (size_t)Pp * GMCO_DVH_K * sizeof(float),
                               cudaMemcpyDefault, m->stream));
        }
        if (T_out && T_out[p]) {
            CK(launch_square(s.x, pr->dTout, Pp, pb.n_dwell, pb.nd_pad, m->stream));
            m->launches++;
            CK(cudaMemcpyAsync(T_out[p], pr->dTout, (size_t)Pp * pb.n_dwell * sizeof(float),
                               cudaMemcpyDefault, m->stream));
        }
        if (objectives && objectives[p])
            CK(cudaMemcpyAsync(objectives[p], s.Ft, (size_t)Pp * sizeof(double), cudaMemcpyDefault,
                               m->stream));
        if (iters_out && iters_out[p])
            CK(cudaMemcpyAsync(iters_out[p], s.iters, (size_t)Pp * sizeof(int32_t),
                               cudaMemcpyDefault, m->stream));
        if (plan_status && plan_status[p])
            CK(cudaMemcpyAsync(plan_status[p], s.status, (size_t)Pp * sizeof(int32_t),
                               cudaMemcpyDefault, m->stream));
    }
    CK(cudaEventRecord(m->ev_out, m->stream));
    CK(cudaStreamWaitEvent((cudaStream_t)cuda_stream, m->ev_out, 0));
    CK(cudaStreamSynchronize(m->stream));
    return rs;
}

gmco_status gmco_multi_autotune_tiles(gmco_multi *m, const float *const *penalty_weights,
                                      const int64_t *P, int32_t steps, const int32_t *split_kb,
                                      const int32_t *grad_plan_tile, int32_t n_candidates,
                                      double *ms_per_step, int32_t *best_index)
{
    std::vector<int64_t> Pv;
    CKS(multi_args(m, penalty_weights, P, &Pv, "gmco_multi_autotune"));
    if (!split_kb || !grad_plan_tile || n_candidates < 1 || n_candidates > 64 || steps < 2 ||
        steps > 1024) {
        set_error_msg("gmco_multi_autotune: bad arguments");
        return GMCO_EINVAL;
    }
    for (int c = 0; c < n_candidates; ++c)
        if (split_kb[c] < 0 ||
            (grad_plan_tile[c] != 0 && grad_plan_tile[c] != 128 && grad_plan_tile[c] != 256)) {
            set_error_msg("gmco_multi_autotune: bad candidate");
            return GMCO_EINVAL;
        }
    CK(cudaSetDevice(m->device));
    const int st = (int)round_up(steps, 2);
    const int32_t saved_split = m->split_kb, saved_tile = m->grad_tile;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    gmco_status rs = GMCO_OK;
    double best_ms = INFINITY;
    int32_t best_c = -1;
    for (int c = 0; c < n_candidates && rs == GMCO_OK; ++c) {
        m->split_kb = split_kb[c];
        m->grad_tile = grad_plan_tile[c];
        if ((rs = multi_workspace(m, Pv)) != GMCO_OK) break;
        if ((rs = multi_graph(m, st, 0.0)) != GMCO_OK) break;
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && rs == GMCO_OK; ++rep) {   // warm-up, then timed
            if ((rs = multi_start(m, penalty_weights, nullptr, 1 << 30)) != GMCO_OK) break;
            if (cudaEventRecord(e0, m->stream) != cudaSuccess ||
                cudaGraphLaunch(m->gexec, m->stream) != cudaSuccess ||
                cudaEventRecord(e1, m->stream) != cudaSuccess ||
                cudaStreamSynchronize(m->stream) != cudaSuccess) {
                set_error("gmco_multi_autotune: timed run", cudaGetLastError());
                rs = GMCO_ECUDA;
                break;
            }
            cudaEventElapsedTime(&ms, e0, e1);
        }
        if (rs != GMCO_OK) break;
        if ((rs = multi_check_err(m)) != GMCO_OK) break;
        const double per = (double)ms / st;
        if (ms_per_step) ms_per_step[c] = per;
        if (per < best_ms) {
            best_ms = per;
            best_c = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs == GMCO_OK && best_c >= 0) {
        m->split_kb = split_kb[best_c];
        m->grad_tile = grad_plan_tile[best_c];
        if (best_index) *best_index = best_c;
    } else {
        m->split_kb = saved_split;
        m->grad_tile = saved_tile;
    }
    return rs;
}

gmco_status gmco_multi_autotune(gmco_multi *m, const float *const *penalty_weights,
                                const int64_t *P, int32_t steps, const int32_t *candidates,
                                int32_t n_candidates, double *ms_per_step, int32_t *best)
{
    if (!m || !candidates || n_candidates < 1 || n_candidates > 64) {
        set_error_msg("gmco_multi_autotune: bad arguments");
        return GMCO_EINVAL;
    }
    const std::vector<int32_t> tiles((size_t)n_candidates, m->grad_tile);
    int32_t bi = -1;
    const gmco_status rs = gmco_multi_autotune_tiles(m, penalty_weights, P, steps, candidates,
                                                     tiles.data(), n_candidates, ms_per_step, &bi);
    if (rs == GMCO_OK && best) *best = candidates[bi];
    return rs;
}

gmco_status gmco_warm_start(gmco_problem *pr, gmco_mlp *mlp, const float *features,
                            const float *penalty_weights, int64_t P, float t_floor,
                            float *t0_out, int32_t *from_model, void *cuda_stream)
{
    if (!pr || !mlp || !features || !penalty_weights || !t0_out || P < 1 || P > (1 << 20) ||
        !(t_floor >= 0.0f) || !isfinite(t_floor)) {
        set_error_msg("gmco_warm_start: bad arguments");
        return GMCO_EINVAL;
    }
    if (pr->pb.n_struct != 4) {
        set_error_msg("gmco_warm_start: the network takes 4 penalty weights per plan");
        return GMCO_EUNSUPPORTED;
    }
    pr->launches = 0;
    CKS(begin_call(pr, cuda_stream));
    CKS(ensure_workspace(pr, (int32_t)P));
    const DevProblem &pb = pr->pb;
    CKS(stage_in(pr, penalty_weights, pr->dW, (size_t)P * pb.n_struct * sizeof(float)));
    int32_t bad = 0;
    CKS(count_bad(pr, pr->dW, P * pb.n_struct, false, &bad));
    if (bad) {
        set_error_msg("gmco_warm_start: negative or non-finite weights");
        return GMCO_EINVAL;
    }
    const gmco_status ms = gmco_mlp_predict(mlp, features, pb.n_dwell, pr->dW, P, t_floor, pr->dT0,
                                            pr->stream);
    if (ms != GMCO_OK) {
        set_error_msg((std::string("gmco_warm_start: ") + gmco_mlp_last_error()).c_str());
        return ms;
    }
    pr->launches += gmco_mlp_last_launch_count(mlp);
    SolverState s = pr->s;
    s.P = (int32_t)P;
    const int form = pr->opt.precision == GMCO_PREC_FP32 ? 0 : 1;
    // objective of the prediction, then of the uniform start
    CK(launch_solver_init(s, pb, pr->dW, pr->dT0, 0, pr->stream));
    CK(launch_compact(s, 0, pr->stream));
    CKS(launch_eval(pr, s, form, false, pr->stream));
    CK(cudaMemcpyAsync(pr->dObj, s.Ft, (size_t)P * sizeof(double), cudaMemcpyDeviceToDevice, pr->stream));
    CK(launch_solver_init(s, pb, pr->dW, nullptr, 0, pr->stream));
    CK(launch_compact(s, 0, pr->stream));
    CKS(launch_eval(pr, s, form, false, pr->stream));
    pr->launches += 4;
    k_choose_start<<<(unsigned)P, 128, 0, pr->stream>>>(pr->dObj, s.Ft, pr->dT0, pb.n_dwell, pr->dTout,
                                                        pr->dIters);
    CK(cudaGetLastError());
    pr->launches++;
    CK(cudaMemcpyAsync(t0_out, pr->dTout, (size_t)P * pb.n_dwell * sizeof(float), cudaMemcpyDefault,
                       pr->stream));
    if (from_model)
        CK(cudaMemcpyAsync(from_model, pr->dIters, (size_t)P * sizeof(int32_t), cudaMemcpyDefault,
                           pr->stream));
    CKS(check_tc_error(pr));
    CKS(end_call(pr, cuda_stream));
    return GMCO_OK;
}

}  // extern "C"
