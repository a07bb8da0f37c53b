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
        int32_t P = -1, form = -1, max_ls = -1, steps = -1, window = -1;
        double tol = -1, c1 = -1;
        bool operator==(const GraphKey &o) const
        {
            return P == o.P && form == o.form && max_ls == o.max_ls && steps == o.steps &&
                   window == o.window && tol == o.tol && c1 == o.c1;
        }
    };
    GraphKey gkey[2];
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};

    int64_t launches = 0;
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
        grows = std::max(grows, max_split_rows(tc_split_plan(pb), cap));
    CK(a.alloc(&pr->gpart, (size_t)grows * pb.nd_pad));
    if (pr->opt.precision != GMCO_PREC_FP32) {
        cudaError_t e = tc_alloc(pb, cap, &pr->tcb, [&](void **p, size_t bytes) {
            unsigned char *q = nullptr;
            cudaError_t r = a.alloc(&q, bytes);
            *p = q;
            return r;
        });
        CK(e);
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
        CK(tc_launch_eval(pb, s, pr->tcb, pr->Fpart, pr->dFpart, pr->gpart, pr->cap, with_dT,
                          nullptr, false, st, &nl, ev));
        pr->launches += nl;
    }
    return GMCO_OK;
}

// Dose-mode FP32 evaluation of every plan at x: doses into pr->G (rows = plans in list
// order), objectives into s.Ft.
gmco_status launch_dose_eval(gmco_problem *pr, cudaStream_t st)
{
    SolverState &s = pr->s;
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
                         cudaStream_t st)
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
            int32_t nl = 0;
            CK(tc_launch_gemms(pb, pr->tcb, cur, pr->Fpart, pr->dFpart, pr->gpart, pr->cap, true,
                               nullptr, st, &nl));
            a.n_ptiles = tc_n_ptiles(pb);
            a.sp = tc_split_plan(pb);
            a.fmt = 1;
            for (int j = 0; j < 3; ++j) a.Tb[j] = pr->tcb.T[j];
            a.dTb = pr->tcb.dT;
            a.nT = std::max(pb.tc_terms, 2);
            a.kpad = (int32_t)pb.kpad;
            a.Wc = pr->tcb.Wc;
        }
        CK(cudaMemsetAsync(next, 0, sizeof(int32_t), st));
        CK(launch_step(s, u, a, st));
    }
    return GMCO_OK;
}

// Runs the step loop with evaluation `form` until every plan is DONE.
gmco_status run_loop(gmco_problem *pr, int form, int32_t P, const UpdateParams &u,
                     int64_t max_steps, int64_t *steps_done)
{
    const int steps = (int)round_up(std::max(2, pr->opt.steps_per_poll), 2);
    // rows of the first step: every plan in INIT or TRIAL, by compaction and preparation
    {
        SolverState s0 = pr->s;
        CK(launch_compact(s0, 0, pr->stream));
        if (form == 0) {
            CK(launch_prep_fp32(s0, pr->pb, pr->Tc, pr->dTc, pr->Wc, false, pr->stream));
        } else {
            CK(tc_launch_prep(pr->pb, s0, pr->tcb, pr->cap, false, pr->stream));
        }
        pr->launches += 2;
    }
    gmco_problem::GraphKey key;
    key.P = P;
    key.form = form;
    key.max_ls = u.max_ls;
    key.steps = steps;
    key.window = u.stop_window;
    key.tol = u.tol;
    key.c1 = u.c1;
    if (!(pr->gkey[form] == key) || !pr->gexec[form]) {
        if (pr->gexec[form]) cudaGraphExecDestroy(pr->gexec[form]);
        pr->gexec[form] = nullptr;
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(pr->stream, cudaStreamCaptureModeThreadLocal));
        const int64_t l0 = pr->launches;
        gmco_status rs = record_steps(pr, form, steps, u, pr->stream);
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
    // launches per graph: steps x (dose GEMM + gradient GEMM + k_step); memsets not counted
    const int64_t per_graph = (int64_t)steps * 3;
    int64_t done = 0;
    for (;;) {
        CK(cudaGraphLaunch(pr->gexec[form], pr->stream));
        pr->launches += per_graph;
        done += steps;
        CK(cudaMemcpyAsync(pr->h_pinned, pr->s.n_act, sizeof(int32_t), cudaMemcpyDeviceToHost,
                           pr->stream));
        CK(cudaStreamSynchronize(pr->stream));
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

}  // namespace

extern "C" {

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
        o.steps_per_poll > 1024 || o.stop_window < 1) {
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
            set_error_msg("gmco_create_problem: tensor-core forms need n_dwell <= 384, n_struct <= 8");
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
    UpdateParams u{pr->opt.c1, tol, pr->opt.max_ls, pr->opt.stop_window};
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
    CKS(launch_dose_eval(pr, pr->stream));
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
            CKS(launch_dose_eval(pr, pr->stream));
        } else {
            CK(launch_compact(s, 1, pr->stream));
            int32_t nl = 0;
            CK(tc_launch_eval(pb, s, pr->tcb, pr->Fpart, pr->dFpart, pr->gpart, pr->cap, false,
                              pr->G, true, pr->stream, &nl));
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

gmco_status gmco_profile_evaluate(gmco_problem *pr, const float *penalty_weights, int64_t P,
                                  const float *X, int32_t reps, double *ms, double *flops)
{
    if (!pr || !penalty_weights || !X || !ms || P < 1 || P > (1 << 20) || reps < 1) {
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
    cudaEvent_t ev[5];
    for (int k = 0; k < 5; ++k) CK(cudaEventCreate(&ev[k]));
    double acc[4] = {0, 0, 0, 0};
    gmco_status rs = GMCO_OK;
    for (int r = 0; r < reps + 1 && rs == GMCO_OK; ++r) {   // first repetition is warm-up
        rs = launch_eval(pr, s, form, true, pr->stream, ev);
        if (rs != GMCO_OK) break;
        if (cudaStreamSynchronize(pr->stream) != cudaSuccess) { rs = GMCO_ECUDA; break; }
        if (r == 0) continue;
        for (int k = 0; k < 4; ++k) {
            float t = 0.0f;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            acc[k] += t;
        }
    }
    for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
    if (rs != GMCO_OK) return rs;
    for (int k = 0; k < 4; ++k) ms[k] = acc[k] / reps;
    if (flops) {
        // algorithmic: dose d and dose change dd (2 contractions), gradient (1 contraction)
        const double c = 2.0 * (double)P * (double)pb.n_pnt * (double)pb.n_dwell;
        flops[0] = 2.0 * c;
        flops[1] = c;
        // issued on the tensor cores (split terms, padded tiles); FP32 form: algorithmic
        if (form == 1) {
            const double cp = 2.0 * (double)round_up(P, 128) * (double)pb.np_pad *
                              (double)round_up(pb.n_dwell, 16);
            flops[2] = tc_mma_units(pb, true, 1) * cp;
            flops[3] = tc_mma_units(pb, true, 2) * cp;
        } else {
            flops[2] = flops[0];
            flops[3] = flops[1];
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

}  // extern "C"
