// Batched L-BFGS machinery (Sec. 2.2.2 of the paper, whose L-BFGS details are omitted there;
// this follows Nocedal & Wright's two-loop recursion with backtracking Armijo search).
//
// Every plan runs the same per-plan state machine; one "step" evaluates every plan that is
// not DONE exactly once:
//   INIT  : evaluate at x0 = sqrt(t0), then choose the first direction
//   TRIAL : evaluate at x + alpha p; accept (Armijo) -> curvature pair, stop test, next
//           direction; or reject -> alpha /= 2 and stay TRIAL
//   DONE  : frozen
// The Armijo and stop tests use dF = F(x + alpha p) - F(x) evaluated from the dose change
// A (t_trial - t), with t_trial - t = alpha p (2 x + alpha p), instead of a difference of
// two rounded objective values (see the evaluation kernels).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace gmco {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Warp reductions as XOR butterflies: every lane ends with the same value (lanes L and L ^ o
// add the same two operands, and addition is commutative), one shuffle fewer than a down-sweep
// plus a broadcast, which matters on the step's serial chains.
__device__ __forceinline__ float warp_sum_f(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ float warp_max_f(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__global__ void k_solver_init(SolverState s, const float *__restrict__ W,
                              const float *__restrict__ t0, const float *__restrict__ inv_count,
                              int32_t nd, int32_t max_iters)
{
    const int j = blockIdx.x;
    if (j >= s.P) return;
    const size_t base = (size_t)j * s.nd_pad;
    for (int l = threadIdx.x; l < s.nd_pad; l += blockDim.x) {
        float xv = 0.0f;
        if (l < nd) xv = t0 ? sqrtf(t0[(size_t)j * nd + l]) : 1.0f;
        s.x[base + l] = xv;
        s.xt[base + l] = xv;
        s.g[base + l] = 0.0f;
        s.gt[base + l] = 0.0f;
        s.p[base + l] = 0.0f;
    }
    if (threadIdx.x < s.n_struct)
        s.Wn[(size_t)j * s.n_struct + threadIdx.x] =
            W[(size_t)j * s.n_struct + threadIdx.x] * inv_count[threadIdx.x];
    if (threadIdx.x == 0) {
        s.state[j] = ST_INIT;
        s.status[j] = GMCO_PLAN_MAXITER;
        s.iters[j] = 0;
        s.maxit[j] = max_iters;
        s.ls[j] = 0;
        s.hcount[j] = 0;
        s.hnewest[j] = s.m - 1;
        s.nsmall[j] = 0;
        s.nevals[j] = 0;
        s.F[j] = 0.0;
        s.Ft[j] = 0.0;
        s.dFt[j] = 0.0;
        s.gtp[j] = 0.0;
        s.alpha[j] = 0.0;
        s.gamma[j] = 1.0;
    }
}

// Single-block stream compaction of the plans that need an evaluation this step, in plan
// order (mode 0: INIT or TRIAL; mode 1: every plan).  Writes list[] and *n_act.
__global__ void k_compact(SolverState s, int32_t mode)
{
    __shared__ int32_t wsum[32];
    const int P = s.P;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int chunk = (P + blockDim.x - 1) / blockDim.x;
    const int b = min(tid * chunk, P), e = min(b + chunk, P);
    int c = 0;
    for (int j = b; j < e; ++j) {
        const int st = s.state[j];
        c += (mode == 1) || st == ST_INIT || st == ST_TRIAL;
    }
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        int v = lane < nw ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v += u;
        }
        if (lane < nw) wsum[lane] = v;  // inclusive warp totals
    }
    __syncthreads();
    int off = incl - c + (wid > 0 ? wsum[wid - 1] : 0);
    for (int j = b; j < e; ++j) {
        const int st = s.state[j];
        if ((mode == 1) || st == ST_INIT || st == ST_TRIAL) s.list[off++] = j;
    }
    if (tid == blockDim.x - 1) *s.n_act = off;
}

// Trial point of each compact row: x_t = x + alpha p and dT = t_t - t = alpha p (2 x + alpha p)
// (rows in INIT or DONE state are evaluated at x itself, dT = 0).  FP32 layout.
__global__ void k_prep_fp32(SolverState s, float *__restrict__ Tc, float *__restrict__ dTc,
                            float *__restrict__ Wc, int32_t force_base)
{
    const int i = blockIdx.x;
    if (i >= *s.n_act) return;
    const int j = s.list[i];
    const bool trial = !force_base && s.state[j] == ST_TRIAL;
    const float a = trial ? (float)s.alpha[j] : 0.0f;
    const size_t pb = (size_t)j * s.nd_pad, cb = (size_t)i * s.nd_pad;
    for (int l = threadIdx.x; l < s.nd_pad; l += blockDim.x) {
        const float xv = s.x[pb + l];
        float xt = xv, dt = 0.0f;
        if (trial) {
            const float ap = a * s.p[pb + l];
            xt = xv + ap;
            dt = ap * (2.0f * xv + ap);
        }
        s.xt[pb + l] = xt;
        Tc[cb + l] = xt * xt;
        if (dTc) dTc[cb + l] = dt;
    }
    if (threadIdx.x < s.n_struct)
        Wc[(size_t)i * s.n_struct + threadIdx.x] = s.Wn[(size_t)j * s.n_struct + threadIdx.x];
    if (threadIdx.x == 0) s.slot_of[j] = i;
}

// gt = 2 x_t * sum_split gpart (chain rule of t = x^2, Eq. (2)); Ft, dFt = fixed-order FP64
// sums of the per-tile partials.
__global__ void k_finish(SolverState s, EvalArgs e, int32_t n_ptiles)
{
    const int i = blockIdx.x;
    if (i >= *e.n_rows) return;
    const int j = s.list[i];
    const int nd = s.nd_pad;
    if (e.gpart) {
        const int R = *e.n_rows;
        int kbps, n_split;
        split_plan(e.sp, R, &kbps, &n_split);
        // split order per element, as in the fused step; up to 8 elements per thread
        // (nd <= 1024 = 8 x 128 threads) loaded independently within each split
        float acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = 0.0f;
        for (int q = 0; q < n_split; ++q) {
            const float *gq = e.gpart + ((size_t)q * R + i) * nd;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int l = threadIdx.x + k * 128;
                if (l < nd) acc[k] += gq[l];
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int l = threadIdx.x + k * 128;
            if (l < nd) s.gt[(size_t)j * nd + l] = 2.0f * s.xt[(size_t)j * nd + l] * acc[k];
        }
    }
    __shared__ double red[2][128];
    double f = 0.0, df = 0.0;
    for (int t = threadIdx.x; t < n_ptiles; t += blockDim.x) {
        f += (double)e.Fpart[(size_t)i * n_ptiles + t];
        if (e.dFpart) df += (double)e.dFpart[(size_t)i * n_ptiles + t];
    }
    red[0][threadIdx.x] = f;
    red[1][threadIdx.x] = df;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        s.Ft[j] = red[0][0];
        s.dFt[j] = red[1][0];
    }
}

__device__ __forceinline__ void plan_done(const SolverState &s, int j, int status, int lane)
{
    if (lane == 0) {
        s.state[j] = ST_DONE;
        s.status[j] = status;
    }
}

// Next trial row of plan j in compact slot `slot`: x_t = x + alpha p, t = x_t^2 and
// dT = alpha p (2 x + alpha p), written in the evaluation form's operand layout.  x and p are
// this lane's elements (lane + 32 e), already in registers.
template <int EPL>
__device__ __forceinline__ void write_trial_row(const SolverState &s, const StepArgs &a, int j,
                                                int slot, float alpha, int lane,
                                                const float (&xv)[EPL], const float (&pv)[EPL])
{
    const int nd = s.nd_pad, epl = nd >> 5;
    const size_t vb = (size_t)j * nd;
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
        if (e >= epl) continue;
        const int l = lane + 32 * e;
        const float ap = alpha * pv[e];
        const float xn = xv[e] + ap;
        const float dt = ap * (2.0f * xv[e] + ap);
        s.xt[vb + l] = xn;
        const float t = xn * xn;
        if (a.fmt == 0) {
            a.Tc[(size_t)slot * nd + l] = t;
            a.dTc[(size_t)slot * nd + l] = dt;
        } else {
            const size_t o = (size_t)slot * a.ldT + l;
            const __nv_bfloat16 t1 = __float2bfloat16_rn(t);
            a.Tb[0][o] = t1;
            const float r1 = t - __bfloat162float(t1);
            if (a.nT > 1) {
                const __nv_bfloat16 t2 = __float2bfloat16_rn(r1);
                a.Tb[1][o] = t2;
                if (a.nT > 2) a.Tb[2][o] = __float2bfloat16_rn(r1 - __bfloat162float(t2));
            }
            const __nv_bfloat16 d1 = __float2bfloat16_rn(dt);
            a.dTb[0][o] = d1;
            a.dTb[1][o] = __float2bfloat16_rn(dt - __bfloat162float(d1));
        }
    }
    if (a.fmt != 0) {   // BF16 rows are kpad long: keep the columns past nd_pad at zero
        for (int l = nd + lane; l < a.kpad; l += 32) {
            const size_t o = (size_t)slot * a.ldT + l;
            for (int k = 0; k < a.nT; ++k) a.Tb[k][o] = __float2bfloat16_rn(0.0f);
            a.dTb[0][o] = __float2bfloat16_rn(0.0f);
            a.dTb[1][o] = __float2bfloat16_rn(0.0f);
        }
    }
    if (lane < s.n_struct)
        a.Wc[(size_t)slot * s.n_struct + lane] = s.Wn[(size_t)j * s.n_struct + lane];
}

// One solver step for plan j (warp per plan), after the evaluation of its compact row:
//   sum the per-tile objective partials and the per-split gradient partials (gt = 2 x_t A^T G),
//   INIT: take F, g; TRIAL: Armijo test on dF (FP64), curvature pair (FP64 s'y, y'y), stop test;
//   new direction by the two-loop recursion; then, if the plan still runs, claim a slot of the
//   next step's compact rows and write its next trial point there.
// The step is one warp's dependent chain, so its global loads are issued together at the start
// (the plan's scalars, rho of every history slot on the lanes, x, p, g, x_t) and the vectors
// stay in registers until the next trial row is written.
// The history rows go to shared memory by bulk copies (the copy engine, one instruction per
// row) tracked by one mbarrier per plan, so that the warp's load/store unit stays free for the
// objective and gradient partials read meanwhile.
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void hbar_init(uint64_t *b)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void hbar_expect(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_to_smem(void *dst, const void *src, uint32_t bytes, uint64_t *b)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(b))
        : "memory");
}
// Waits (every lane) for the barrier's first phase; gives up after about a second.
__device__ __forceinline__ bool hbar_wait(uint64_t *b)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(b))
            : "memory");
        if (done) return true;
        if (clock64() - t0 > 2000000000LL) return false;
    }
}

// hS / hY: this plan's history rows in shared memory (m x nd each, the same slots as s.S / s.Y),
// or null to read them from global memory
// hbar: with hS, the mbarrier of the bulk history copies; *hbar_used is set once they are
// issued (the caller then waits for them before the block exits).
template <int EPL, bool ONE_TRIP = false>
__device__ __forceinline__ void step_plan(const SolverState &s, const UpdateParams &u,
                                          const StepArgs &a, const int j, const int lane,
                                          float *hS = nullptr, float *hY = nullptr,
                                          uint64_t *hbar = nullptr, bool *hbar_used = nullptr)
{
    const int nd = s.nd_pad, epl = nd >> 5, m = s.m;
    const size_t vb = (size_t)j * nd;
    // the plan's scalars, read by every lane before lane 0 writes any of them
    const int st = s.state[j];
    int it = s.iters[j];
    int cnt = s.hcount[j];
    int nw = s.hnewest[j];
    const double F_old = s.F[j];
    const int nsmall_old = s.nsmall[j];
    const double alpha_old = s.alpha[j], gtp_old = s.gtp[j];
    const int ls_old = s.ls[j];
    const int maxit = s.maxit[j];
    const int ne = s.nevals[j] + 1;   // this evaluation included
    const int slot = s.slot_of[j];
    const int R = *a.rows_cur;
    double rho_l = lane < m ? s.rho[(size_t)j * m + lane] : 0.0;   // lane i: rho of slot i
    double gam = s.gamma[j];
    __syncwarp();
    if (st != ST_INIT && st != ST_TRIAL) return;
    if (lane == 0) s.nevals[j] = ne;
    float *x = s.x + vb, *g = s.g + vb, *p = s.p + vb;
    const float *xt = s.xt + vb;
    float xv[EPL], pv[EPL], gov[EPL], xtv[EPL];
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
        const int l = lane + 32 * e;
        xv[e] = e < epl ? x[l] : 0.0f;
        pv[e] = e < epl ? p[l] : 0.0f;
        gov[e] = e < epl ? g[l] : 0.0f;
        xtv[e] = e < epl ? xt[l] : 0.0f;
    }
    // the history rows the two-loop will read, copied asynchronously while the partial sums
    // below are added (16-byte copies; rows are nd_pad floats, a multiple of 32)
    const float *HS = s.S + (size_t)j * m * nd, *HY = s.Y + (size_t)j * m * nd;
    const float *HSg = HS, *HYg = HY;   // the global rows, kept for a wait that gives up
    if (hS) {   // rows of nd_pad floats: 16-byte aligned, a multiple of 16 bytes
        if (lane == 0) {
            hbar_expect(hbar, (uint32_t)cnt * 2u * (uint32_t)nd * 4u);
            if (cnt == m) {   // a full ring is contiguous here and there: one copy each for s and y
                bulk_to_smem(hS, HS, (uint32_t)m * (uint32_t)nd * 4u, hbar);
                bulk_to_smem(hY, HY, (uint32_t)m * (uint32_t)nd * 4u, hbar);
            } else {
                for (int k = 0, i = nw; k < cnt; ++k, i = i == 0 ? m - 1 : i - 1) {   // newest first
                    bulk_to_smem(hS + (size_t)i * nd, HS + (size_t)i * nd, (uint32_t)nd * 4u, hbar);
                    bulk_to_smem(hY + (size_t)i * nd, HY + (size_t)i * nd, (uint32_t)nd * 4u, hbar);
                }
            }
        }
        *hbar_used = true;
        HS = hS;
        HY = hY;
    }
    // every copy into shared memory has landed; if a bulk copy's wait gave up (never expected),
    // the history is read from global memory instead and shared memory is left alone
    bool staged = hS != nullptr;
    auto history_ready = [&]() {
        if (!staged) return;
        if (!__all_sync(kFull, hbar_wait(hbar))) {
            staged = false;
            HS = HSg;
            HY = HYg;
        }
        __syncwarp();
    };

    // ---- results of this step's evaluation (fixed summation order)
    double fsum = 0.0, dfsum = 0.0;
#pragma unroll 4
    for (int t = lane; t < a.n_ptiles; t += 32) {
        fsum += (double)a.Fpart[(size_t)slot * a.n_ptiles + t];   // a row's partials are contiguous
        if (st == ST_TRIAL) dfsum += (double)a.dFpart[(size_t)slot * a.n_ptiles + t];
    }
    const double Ft = warp_sum_d(fsum);
    const double dF = warp_sum_d(dfsum);
    int kbps, n_split;
    split_plan(a.sp, R, &kbps, &n_split);
    if (a.sp_flag && *a.sp_flag) n_split = 1;
    // sum over the splits in split order; each split's EPL loads are independent, so the
    // latency chain is one load per batch of splits rather than one per element and split
    float gtv[EPL];
#pragma unroll
    for (int e = 0; e < EPL; ++e) gtv[e] = 0.0f;
    constexpr int QB = EPL <= 12 ? 8 : 4;   // splits in flight (registers: QB x EPL)
    int q = 0;
    if constexpr (ONE_TRIP) {
        // the last, partial batch of splits as one masked round trip (the single-problem
        // kernel has the registers for it; the multi-problem one would spill)
        for (; q < n_split; q += QB) {
            float v[QB][EPL];
#pragma unroll
            for (int r = 0; r < QB; ++r) {
                const bool on = q + r < n_split;
                const float *gq = a.gpart + ((size_t)(on ? q + r : q) * R + slot) * nd + lane;
#pragma unroll
                for (int e = 0; e < EPL; ++e) v[r][e] = on && e < epl ? gq[32 * e] : 0.0f;
            }
#pragma unroll
            for (int r = 0; r < QB; ++r)
#pragma unroll
                for (int e = 0; e < EPL; ++e)
                    if (e < epl && q + r < n_split) gtv[e] += v[r][e];
        }
    }
    for (; q + QB <= n_split; q += QB) {
        float v[QB][EPL];
#pragma unroll
        for (int r = 0; r < QB; ++r) {
            const float *gq = a.gpart + ((size_t)(q + r) * R + slot) * nd + lane;
#pragma unroll
            for (int e = 0; e < EPL; ++e) v[r][e] = e < epl ? gq[32 * e] : 0.0f;
        }
#pragma unroll
        for (int r = 0; r < QB; ++r)
#pragma unroll
            for (int e = 0; e < EPL; ++e)
                if (e < epl) gtv[e] += v[r][e];
    }
    for (; q < n_split; ++q) {
        const float *gq = a.gpart + ((size_t)q * R + slot) * nd + lane;
#pragma unroll
        for (int e = 0; e < EPL; ++e)
            if (e < epl) gtv[e] += gq[32 * e];
    }
#pragma unroll
    for (int e = 0; e < EPL; ++e)
        if (e < epl) gtv[e] *= 2.0f * xtv[e];

    float gv[EPL];
    float gmax = 0.0f;
    bool need_dir = false;
    double alpha_next = 0.0;

    if (st == ST_INIT) {
        bool fin = isfinite(Ft);
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
            gv[e] = 0.0f;
            if (e < epl) {
                gv[e] = gtv[e];
                g[lane + 32 * e] = gv[e];
                fin = fin && isfinite(gv[e]);
                gmax = fmaxf(gmax, fabsf(gv[e]));
            }
        }
        fin = __all_sync(kFull, fin);
        gmax = warp_max_f(gmax);
        if (lane == 0) {
            s.F[j] = Ft;
            s.Ft[j] = Ft;
        }
        if (!fin) { plan_done(s, j, GMCO_PLAN_NONFINITE, lane); return; }
        if (Ft == 0.0 || gmax == 0.0f) { plan_done(s, j, GMCO_PLAN_CONVERGED, lane); return; }
        need_dir = true;
    } else {
        const double alpha = alpha_old, gtp = gtp_old;
        const bool ok = isfinite(dF) && isfinite(Ft) && dF <= u.c1 * alpha * gtp;
        if (ok) {
            float sv[EPL], yv[EPL];
            double sy = 0.0, yy = 0.0, sy1 = 0.0, yy1 = 0.0;   // two partial sums each
            bool fin = true;
#pragma unroll
            for (int e = 0; e < EPL; ++e) {
                sv[e] = 0.0f;
                yv[e] = 0.0f;
                gv[e] = 0.0f;
                if (e < epl) {
                    const int l = lane + 32 * e;
                    const float xn = xtv[e], gn = gtv[e];
                    sv[e] = xn - xv[e];
                    yv[e] = gn - gov[e];
                    if (e & 1) {
                        sy1 += (double)sv[e] * (double)yv[e];
                        yy1 += (double)yv[e] * (double)yv[e];
                    } else {
                        sy += (double)sv[e] * (double)yv[e];
                        yy += (double)yv[e] * (double)yv[e];
                    }
                    fin = fin && isfinite(gn);
                    gmax = fmaxf(gmax, fabsf(gn));
                    x[l] = xn;
                    g[l] = gn;
                    xv[e] = xn;
                    gv[e] = gn;
                }
            }
            sy = warp_sum_d(sy + sy1);   // curvature products in FP64
            yy = warp_sum_d(yy + yy1);
            fin = __all_sync(kFull, fin);
            gmax = warp_max_f(gmax);
            if (fin && sy > 1e-12 * yy) {
                nw = nw + 1 == m ? 0 : nw + 1;
                float *Sd = s.S + ((size_t)j * m + nw) * nd;
                float *Yd = s.Y + ((size_t)j * m + nw) * nd;
                history_ready();   // the copy of the slot being replaced has landed
#pragma unroll
                for (int e = 0; e < EPL; ++e)
                    if (e < epl) {
                        Sd[lane + 32 * e] = sv[e];
                        Yd[lane + 32 * e] = yv[e];
                        if (staged) {
                            hS[(size_t)nw * nd + lane + 32 * e] = sv[e];
                            hY[(size_t)nw * nd + lane + 32 * e] = yv[e];
                        }
                    }
                cnt = min(cnt + 1, m);
                const double rho_new = __drcp_rn(sy);   // 1 / sy, correctly rounded
                gam = sy / yy;
                if (lane == nw) rho_l = rho_new;
                if (lane == 0) {
                    s.rho[(size_t)j * m + nw] = rho_new;
                    s.gamma[j] = gam;
                }
                if (staged) __syncwarp();   // the new pair is read back by every lane below
            }
            const double Fprev = F_old;
            ++it;
            if (lane == 0) {
                s.F[j] = Fprev + dF;
                s.Ft[j] = Ft;
                s.iters[j] = it;
                s.hcount[j] = cnt;
                s.hnewest[j] = nw;
            }
            if (!fin) { plan_done(s, j, GMCO_PLAN_NONFINITE, lane); return; }
            const int nsm = fabs(dF) <= u.tol * fmax(fabs(Fprev), 1e-300) ? nsmall_old + 1 : 0;
            if (lane == 0) s.nsmall[j] = nsm;
            if (Ft == 0.0 || gmax == 0.0f || nsm >= u.stop_window) {
                plan_done(s, j, GMCO_PLAN_CONVERGED, lane);
                return;
            }
            need_dir = true;
        } else {
            const int lsn = ls_old + 1;
            if (lsn >= u.max_ls) {
                if (cnt > 0) {   // retry once along steepest descent with a fresh history
                    cnt = 0;
                    need_dir = true;
#pragma unroll
                    for (int e = 0; e < EPL; ++e) {
                        gv[e] = 0.0f;
                        if (e < epl) {
                            gv[e] = gov[e];
                            gmax = fmaxf(gmax, fabsf(gv[e]));
                        }
                    }
                    gmax = warp_max_f(gmax);
                    if (lane == 0) s.hcount[j] = 0;
                } else {
                    plan_done(s, j, GMCO_PLAN_LSFAIL, lane);
                    return;
                }
            } else {
                alpha_next = alpha * 0.5;
                if (lane == 0) {
                    s.alpha[j] = alpha_next;
                    s.ls[j] = lsn;
                }
            }
        }
    }
    // iteration cap, or the evaluation budget (the next trial would exceed it): stop at x
    if ((need_dir && it >= maxit) || (u.max_evals > 0 && ne >= u.max_evals)) {
        plan_done(s, j, GMCO_PLAN_MAXITER, lane);
        return;
    }

    // the plan runs on: claim its row of the next step now, so that the atomic's round trip
    // overlaps the two-loop below
    int ns = 0;
    if (lane == 0) ns = atomicAdd(a.rows_next, 1);

    if (need_dir) {
        // two-loop recursion, q in registers (FP32 vectors and dot products); the next
        // history pair is loaded while the current dot product is reduced
        float q[EPL];
#pragma unroll
        for (int e = 0; e < EPL; ++e) q[e] = gv[e];
        history_ready();
        if (cnt > 0) {
            // The history loops stay rolled (their bodies are reused from the instruction
            // cache; fully unrolled, one warp's pass over straight-line code is fetch-bound)
            // and alpha_k of the first loop is kept on lane k for the second.
            float al_l = 0.0f;
            const float rho_f = (float)rho_l;   // lane i: rho of slot i, one shuffle per use
            float sc[EPL], yc[EPL];
            {
                const int i0 = nw;
                const float *Si = HS + (size_t)i0 * nd;
                const float *Yi = HY + (size_t)i0 * nd;
#pragma unroll
                for (int e = 0; e < EPL; ++e) {
                    sc[e] = e < epl ? Si[lane + 32 * e] : 0.0f;
                    yc[e] = e < epl ? Yi[lane + 32 * e] : 0.0f;
                }
            }
            int i = nw;   // slot of pair k (newest first); no integer division in the loop
#pragma unroll 1
            for (int k = 0; k < cnt; ++k) {
                float sn[EPL], yn[EPL];
                const bool more = k + 1 < cnt;
                const int i1 = i == 0 ? m - 1 : i - 1;
                const float *Sn = HS + (size_t)i1 * nd;
                const float *Yn = HY + (size_t)i1 * nd;
#pragma unroll
                for (int e = 0; e < EPL; ++e) {
                    sn[e] = (more && e < epl) ? Sn[lane + 32 * e] : 0.0f;
                    yn[e] = (more && e < epl) ? Yn[lane + 32 * e] : 0.0f;
                }
                const float rho = __shfl_sync(kFull, rho_f, i);
                float d0 = 0.0f, d1 = 0.0f;   // two partial sums: half the dependent chain
#pragma unroll
                for (int e = 0; e < EPL; e += 2) {
                    d0 += sc[e] * q[e];
                    if (e + 1 < EPL) d1 += sc[e + 1] * q[e + 1];
                }
                const float av = rho * warp_sum_f(d0 + d1);
                if (lane == k) al_l = av;
#pragma unroll
                for (int e = 0; e < EPL; ++e) {
                    q[e] -= av * yc[e];
                    sc[e] = sn[e];
                    yc[e] = yn[e];
                }
                i = i1;
            }
            const float gamf = (float)gam;
#pragma unroll
            for (int e = 0; e < EPL; ++e) q[e] *= gamf;
            const int io = nw - (cnt - 1) < 0 ? nw - (cnt - 1) + m : nw - (cnt - 1);   // oldest pair first
            {
                const float *Si = HS + (size_t)io * nd;
                const float *Yi = HY + (size_t)io * nd;
#pragma unroll
                for (int e = 0; e < EPL; ++e) {
                    sc[e] = e < epl ? Si[lane + 32 * e] : 0.0f;
                    yc[e] = e < epl ? Yi[lane + 32 * e] : 0.0f;
                }
            }
            i = io;
#pragma unroll 1
            for (int k = cnt - 1; k >= 0; --k) {
                float sn[EPL], yn[EPL];
                const bool more = k > 0;
                const int i1 = i == m - 1 ? 0 : i + 1;
                const float *Sn = HS + (size_t)i1 * nd;
                const float *Yn = HY + (size_t)i1 * nd;
#pragma unroll
                for (int e = 0; e < EPL; ++e) {
                    sn[e] = (more && e < epl) ? Sn[lane + 32 * e] : 0.0f;
                    yn[e] = (more && e < epl) ? Yn[lane + 32 * e] : 0.0f;
                }
                const float rho = __shfl_sync(kFull, rho_f, i);
                const float alk = __shfl_sync(kFull, al_l, k);
                float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
                for (int e = 0; e < EPL; e += 2) {
                    d0 += yc[e] * q[e];
                    if (e + 1 < EPL) d1 += yc[e + 1] * q[e + 1];
                }
                const float b = rho * warp_sum_f(d0 + d1);
#pragma unroll
                for (int e = 0; e < EPL; ++e) {
                    q[e] += sc[e] * (alk - b);
                    sc[e] = sn[e];
                    yc[e] = yn[e];
                }
                i = i1;
            }
        }
        double gtp = 0.0, gtp1 = 0.0;   // two partial sums: half the chain of FP64 adds
#pragma unroll
        for (int e = 0; e < EPL; ++e)
            if (e < epl) {
                if (e & 1) gtp1 += (double)gv[e] * (double)(-q[e]);
                else gtp += (double)gv[e] * (double)(-q[e]);
            }
        gtp = warp_sum_d(gtp + gtp1);   // directional derivative for the Armijo test, FP64
        double alpha0 = (cnt == 0) ? fmin(1.0, 1.0 / (double)gmax) : 1.0;
        if (!(gtp < 0.0)) {       // not a descent direction: steepest descent, fresh history
            cnt = 0;
            double gg = 0.0;
#pragma unroll
            for (int e = 0; e < EPL; ++e) {
                q[e] = gv[e];
                if (e < epl) gg += (double)gv[e] * (double)gv[e];
            }
            gtp = -warp_sum_d(gg);
            alpha0 = fmin(1.0, 1.0 / (double)gmax);
        }
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
            pv[e] = -q[e];
            if (e < epl) p[lane + 32 * e] = pv[e];
        }
        if (lane == 0) {
            s.gtp[j] = gtp;
            s.alpha[j] = alpha0;
            s.ls[j] = 0;
            s.hcount[j] = cnt;
            s.state[j] = ST_TRIAL;
        }
        alpha_next = alpha0;
    }

    // next trial point into the claimed slot of the next step's rows
    ns = __shfl_sync(kFull, ns, 0);
    if (lane == 0) s.slot_of[j] = ns;
    write_trial_row<EPL>(s, a, j, ns, (float)alpha_next, lane, xv, pv);
}

// use_smem: each warp's plan keeps its history rows in dynamic shared memory (2 m nd_pad
// floats per warp)
template <int EPL>
__global__ void __launch_bounds__(256) k_step(SolverState s, UpdateParams u, StepArgs a,
                                              int32_t use_smem)
{
    extern __shared__ __align__(16) float hist[];
    __shared__ __align__(8) uint64_t hbar;   // bulk history copies (one plan per block)
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= s.P) return;
    float *hS = nullptr, *hY = nullptr;
    if (use_smem) {
        hS = hist + (size_t)(threadIdx.x >> 5) * 2 * s.m * s.nd_pad;
        hY = hS + (size_t)s.m * s.nd_pad;
        if ((threadIdx.x & 31) == 0) hbar_init(&hbar);
        __syncwarp();
    }
    bool used = false;
    step_plan<EPL, true>(s, u, a, j, threadIdx.x & 31, hS, hY, use_smem ? &hbar : nullptr, &used);
    if (used) hbar_wait(&hbar);   // nothing in flight into shared memory at exit
}

// The same step for the plans of several problems; each block's problem descriptor is
// staged in shared memory.
template <int EPL>
__global__ void __launch_bounds__(256) k_step_multi(const StepDesc *__restrict__ d,
                                                    const int32_t *__restrict__ block_start,
                                                    int32_t n, UpdateParams u)
{
    __shared__ __align__(16) StepDesc sd;
    __shared__ int32_t s_p;
    const int b = blockIdx.x;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n - 1;   // last p with block_start[p] <= b
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (block_start[mid] <= b) lo = mid; else hi = mid - 1;
        }
        s_p = lo;
    }
    __syncthreads();
    const int p = s_p;
    {
        static_assert(sizeof(StepDesc) % 4 == 0, "descriptor size");
        const uint32_t *src = reinterpret_cast<const uint32_t *>(d + p);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sd);
        for (int i = threadIdx.x; i < (int)(sizeof(StepDesc) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int j = (b - block_start[p]) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= sd.s.P) return;
    step_plan<EPL>(sd.s, u, sd.a, j, threadIdx.x & 31);
}

__global__ void k_sum_counters(int32_t *const *__restrict__ c, int32_t n, int32_t *__restrict__ sum)
{
    int v = 0;
    for (int p = threadIdx.x; p < n; p += 32) v += *c[p];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if (threadIdx.x == 0) *sum = v;
}

// Measurement set-up: every plan in a line-search trial at x + 0.01 x (t_trial != t).
__global__ void k_profile_setup(SolverState s)
{
    const int j = blockIdx.x;
    if (j >= s.P) return;
    for (int l = threadIdx.x; l < s.nd_pad; l += blockDim.x)
        s.p[(size_t)j * s.nd_pad + l] = s.x[(size_t)j * s.nd_pad + l];
    if (threadIdx.x == 0) {
        s.state[j] = ST_TRIAL;
        s.alpha[j] = 0.01;
    }
}

// Re-open finished plans for further iterations (FP32 refinement after a BF16/FP8 solve).
__global__ void k_reopen(SolverState s, int32_t extra)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= s.P) return;
    if (s.state[j] == ST_DONE && s.status[j] != GMCO_PLAN_NONFINITE) {
        s.state[j] = ST_INIT;
        s.status[j] = GMCO_PLAN_MAXITER;
        s.maxit[j] = s.iters[j] + extra;
        s.nsmall[j] = 0;
        s.nevals[j] = 0;   // the refinement has its own evaluation budget
    }
}

__global__ void k_square(const float *__restrict__ x, float *__restrict__ t, int64_t rows,
                         int64_t nd, int64_t nd_pad)
{
    const int64_t n = rows * nd;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = k / nd, l = k - r * nd;
        const float v = x[r * nd_pad + l];
        t[k] = v * v;
    }
}

}  // namespace

cudaError_t launch_solver_init(const SolverState &s, const DevProblem &pb, const float *W,
                               const float *t0, int32_t max_iters, cudaStream_t st)
{
    k_solver_init<<<s.P, 128, 0, st>>>(s, W, t0, pb.inv_count, (int32_t)pb.n_dwell, max_iters);
    return cudaGetLastError();
}

cudaError_t launch_compact(const SolverState &s, int32_t mode, cudaStream_t st)
{
    k_compact<<<1, 1024, 0, st>>>(s, mode);
    return cudaGetLastError();
}

cudaError_t launch_prep_fp32(const SolverState &s, const DevProblem &pb, float *Tc, float *dTc,
                             float *Wc, bool force_base, cudaStream_t st)
{
    (void)pb;
    k_prep_fp32<<<s.P, 128, 0, st>>>(s, Tc, dTc, Wc, force_base ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_finish(const SolverState &s, const EvalArgs &e, int32_t n_ptiles,
                          cudaStream_t st)
{
    k_finish<<<s.P, 128, 0, st>>>(s, e, n_ptiles);
    return cudaGetLastError();
}

constexpr int kStepSmem = 96 * 1024;

cudaError_t step_attrs()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_step<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStepSmem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_step<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStepSmem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_step<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStepSmem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_step<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStepSmem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_step<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStepSmem)) != cudaSuccess) return e;
    done = true;
    return cudaSuccess;
}

cudaError_t launch_step(const SolverState &s, const UpdateParams &u, const StepArgs &a,
                        cudaStream_t st)
{
    // One plan per block with its history rows staged in shared memory when they fit (up to
    // kStepSmem bytes; several blocks share an SM), else two plans per block reading the
    // history from global memory.
    const int epl = s.nd_pad / 32;
    const size_t hist = (size_t)2 * s.m * s.nd_pad * sizeof(float);
    const int use = hist <= (size_t)kStepSmem ? 1 : 0;
    const int tpb = use ? 32 : 64;
    const size_t smem = use ? hist : 0;
    const int blocks = (int)ceil_div((int64_t)s.P * 32, tpb);
    cudaError_t e = step_attrs();
    if (e != cudaSuccess) return e;
    if (epl <= 4) k_step<4><<<blocks, tpb, smem, st>>>(s, u, a, use);
    else if (epl <= 8) k_step<8><<<blocks, tpb, smem, st>>>(s, u, a, use);
    else if (epl <= 12) k_step<12><<<blocks, tpb, smem, st>>>(s, u, a, use);
    else if (epl <= 16) k_step<16><<<blocks, tpb, smem, st>>>(s, u, a, use);
    else k_step<32><<<blocks, tpb, smem, st>>>(s, u, a, use);
    return cudaGetLastError();
}

cudaError_t launch_step_multi(const StepDesc *d, const int32_t *block_start, int32_t n,
                              int32_t total_blocks, int32_t max_nd_pad, const UpdateParams &u,
                              cudaStream_t st)
{
    const int epl = max_nd_pad / 32;
    if (epl <= 4) k_step_multi<4><<<total_blocks, 256, 0, st>>>(d, block_start, n, u);
    else if (epl <= 8) k_step_multi<8><<<total_blocks, 256, 0, st>>>(d, block_start, n, u);
    else if (epl <= 12) k_step_multi<12><<<total_blocks, 256, 0, st>>>(d, block_start, n, u);
    else if (epl <= 16) k_step_multi<16><<<total_blocks, 256, 0, st>>>(d, block_start, n, u);
    else return cudaErrorInvalidValue;   // multi-problem launches serve n_dwell <= 512
    return cudaGetLastError();
}

cudaError_t launch_sum_counters(int32_t *const *counters, int32_t n, int32_t *sum, cudaStream_t st)
{
    k_sum_counters<<<1, 32, 0, st>>>(counters, n, sum);
    return cudaGetLastError();
}

cudaError_t launch_profile_setup(const SolverState &s, cudaStream_t st)
{
    k_profile_setup<<<s.P, 128, 0, st>>>(s);
    return cudaGetLastError();
}

cudaError_t launch_reopen(const SolverState &s, int32_t extra_iters, cudaStream_t st)
{
    k_reopen<<<(int)ceil_div(s.P, 256), 256, 0, st>>>(s, extra_iters);
    return cudaGetLastError();
}

cudaError_t launch_square(const float *x, float *t, int64_t rows, int64_t nd, int64_t nd_pad,
                          cudaStream_t st)
{
    const int64_t n = rows * nd;
    const int blocks = (int)std::min<int64_t>(ceil_div(n, 256), 148 * 16);
    if (n == 0) return cudaSuccess;
    k_square<<<blocks, 256, 0, st>>>(x, t, rows, nd, nd_pad);
    return cudaGetLastError();
}

}  // namespace gmco
