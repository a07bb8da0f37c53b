// FP32 evaluation of Eq. (dose), Eq. (1), Eq. (obj) and Eq. (2) for a batch of plans on the
// SIMT FP32 pipes (the FP32 precision form).
//
// GEMM1  D_t = T_t A^T and dD = dT A^T      (rows = plans, columns = points, K = dwells)
//        epilogue per (plan, point): penalty f (Eq. (1)), its dose derivative, and
//        f(d_t) - f(d_t - dD) in factored form; per-plan sums over the tile's points.
// GEMM2  gpart = G A over a range of points  (rows = plans, columns = dwells, split-K)
//
// Tiles: GEMM1 64 plans x 128 points, GEMM2 64 plans x 128 dwells, K slabs of 16,
// 256 threads each computing 4 x 8 outputs, register double-buffered global loads.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace gmco {

namespace {

constexpr int BM = 64, BN = 128, BK = 16, NT = 256;
constexpr int SP = BM + 4;   // padded shared stride of the plan-row operand

// Penalty of Eq. (1) and its derivative in d, scaled by c = w_ps / N_s.
__device__ __forceinline__ void penalty(float d, float4 prm, float c, float &f, float &df)
{
    const float u = prm.y - d;   // D_min - d
    const float o = d - prm.z;   // d - D_max
    f = 0.0f;
    df = 0.0f;
    if (u > 0.0f) {
        f = c * prm.x * u * u;
        df = -2.0f * c * prm.x * u;
    } else if (o > 0.0f) {
        f = c * prm.w * o * o;
        df = 2.0f * c * prm.w * o;
    }
}

// f(d_t) - f(d_b) with d_b = d_t - dd, without subtracting two rounded penalties:
// u_t^2 - u_b^2 = (u_t - u_b)(u_t + u_b) with u_t - u_b = -dd on the lower side and
// o_t - o_b = dd on the upper side.
__device__ __forceinline__ float penalty_delta(float dt, float dd, float4 prm, float c)
{
    const float db = dt - dd;
    float lo = 0.0f, up = 0.0f;
    const float ut = prm.y - dt, ub = prm.y - db;
    if (ut > 0.0f && ub > 0.0f) lo = -dd * (ut + ub);
    else if (ut > 0.0f) lo = ut * ut;
    else if (ub > 0.0f) lo = -ub * ub;
    const float ot = dt - prm.z, ob = db - prm.z;
    if (ot > 0.0f && ob > 0.0f) up = dd * (ot + ob);
    else if (ot > 0.0f) up = ot * ot;
    else if (ob > 0.0f) up = -ob * ob;
    return c * (prm.x * lo + prm.w * up);
}

template <bool HAS_DT>
__global__ void __launch_bounds__(NT, 2) k_gemm1(EvalArgs e, int32_t mode)
{
    __shared__ __align__(16) float Ts[2][BK][SP];
    __shared__ __align__(16) float dTs[HAS_DT ? 2 : 1][BK][HAS_DT ? SP : 4];
    __shared__ __align__(16) float As[2][BK][BN];
    __shared__ float4 sprm[kMaxStruct];
    __shared__ float sW[BM][kMaxStruct];

    const int n_rows = *e.n_rows;
    const int row0 = blockIdx.y * BM;
    if (row0 >= n_rows) return;
    const int pt0 = blockIdx.x * BN;
    const DevProblem &pb = e.pb;
    const int nd = (int)pb.nd_pad;
    const int S = pb.n_struct;
    const int tid = threadIdx.x;
    const int tr = tid >> 4, tc = tid & 15;

    if (tid < S) sprm[tid] = pb.sparams[tid];
    for (int k = tid; k < BM * S; k += NT) {
        const int r = k / S, s = k - r * S;
        sW[r][s] = (row0 + r < n_rows) ? e.Wc[(size_t)(row0 + r) * S + s] : 0.0f;
    }

    // global load mapping
    const int lr = tid >> 2, lk = (tid & 3) * 4;           // T/dT: row, k offset
    const bool row_ok = row0 + lr < n_rows;
    const float *Tp = e.Tt + (size_t)(row0 + lr) * nd + lk;
    const float *dTp = HAS_DT ? e.dT + (size_t)(row0 + lr) * nd + lk : nullptr;
    const float *Ap0 = pb.A32 + (size_t)(pt0 + lr) * nd + lk;
    const float *Ap1 = pb.A32 + (size_t)(pt0 + lr + 64) * nd + lk;

    float4 rT, rdT, rA0, rA1;
    auto gload = [&](int k0) {
        rT = row_ok ? *reinterpret_cast<const float4 *>(Tp + k0) : make_float4(0, 0, 0, 0);
        if (HAS_DT)
            rdT = row_ok ? *reinterpret_cast<const float4 *>(dTp + k0) : make_float4(0, 0, 0, 0);
        rA0 = *reinterpret_cast<const float4 *>(Ap0 + k0);
        rA1 = *reinterpret_cast<const float4 *>(Ap1 + k0);
    };
    auto sstore = [&](int buf) {
        Ts[buf][lk + 0][lr] = rT.x; Ts[buf][lk + 1][lr] = rT.y;
        Ts[buf][lk + 2][lr] = rT.z; Ts[buf][lk + 3][lr] = rT.w;
        if (HAS_DT) {
            dTs[buf][lk + 0][lr] = rdT.x; dTs[buf][lk + 1][lr] = rdT.y;
            dTs[buf][lk + 2][lr] = rdT.z; dTs[buf][lk + 3][lr] = rdT.w;
        }
        As[buf][lk + 0][lr] = rA0.x; As[buf][lk + 1][lr] = rA0.y;
        As[buf][lk + 2][lr] = rA0.z; As[buf][lk + 3][lr] = rA0.w;
        As[buf][lk + 0][lr + 64] = rA1.x; As[buf][lk + 1][lr + 64] = rA1.y;
        As[buf][lk + 2][lr + 64] = rA1.z; As[buf][lk + 3][lr + 64] = rA1.w;
    };

    float acc[4][8], dacc[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) { acc[r][c] = 0.0f; dacc[r][c] = 0.0f; }

    const int nk = nd / BK;
    gload(0);
    sstore(0);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) gload((kt + 1) * BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 t = *reinterpret_cast<const float4 *>(&Ts[buf][k][tr * 4]);
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][tc * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][64 + tc * 4]);
            const float tv[4] = {t.x, t.y, t.z, t.w};
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(tv[r], av[c], acc[r][c]);
            if (HAS_DT) {
                const float4 d = *reinterpret_cast<const float4 *>(&dTs[buf][k][tr * 4]);
                const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) dacc[r][c] = fmaf(dv[r], av[c], dacc[r][c]);
            }
        }
        if (kt + 1 < nk) sstore(buf ^ 1);
        __syncthreads();
    }

    // epilogue: penalties, derivative, partial sums per plan over this tile's points
    float fs[4] = {0, 0, 0, 0}, dfs[4] = {0, 0, 0, 0};
    int8_t sc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int n = pt0 + (c < 4 ? tc * 4 + c : 64 + tc * 4 + (c - 4));
        sc[c] = pb.sid[n];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int row = row0 + tr * 4 + r;
        float out[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            out[c] = 0.0f;
            const int s = sc[c];
            if (s >= 0) {
                const float4 prm = sprm[s];
                const float cw = sW[tr * 4 + r][s];
                float f, df;
                penalty(acc[r][c], prm, cw, f, df);
                fs[r] += f;
                out[c] = (mode == MODE_DOSE) ? acc[r][c] : df;
                if (HAS_DT) dfs[r] += penalty_delta(acc[r][c], dacc[r][c], prm, cw);
            }
        }
        if (row < n_rows) {
            float *Gr = e.G + (size_t)row * pb.np_pad + pt0;
            *reinterpret_cast<float4 *>(Gr + tc * 4) = make_float4(out[0], out[1], out[2], out[3]);
            *reinterpret_cast<float4 *>(Gr + 64 + tc * 4) =
                make_float4(out[4], out[5], out[6], out[7]);
        }
    }
    // reduce over the 16 column groups (lanes tc = 0..15 of each half-warp), fixed order
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        float v = fs[r], dv = dfs[r];
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            v += __shfl_down_sync(0xffffffffu, v, o, 16);
            dv += __shfl_down_sync(0xffffffffu, dv, o, 16);
        }
        const int row = row0 + tr * 4 + r;
        if (tc == 0 && row < n_rows) {
            e.Fpart[(size_t)row * gridDim.x + blockIdx.x] = v;   // [row][point tile]
            if (e.dFpart) e.dFpart[(size_t)row * gridDim.x + blockIdx.x] = HAS_DT ? dv : 0.0f;
        }
    }
}

__global__ void __launch_bounds__(NT, 2) k_gemm2(EvalArgs e)
{
    __shared__ __align__(16) float Gs[2][BK][SP];
    __shared__ __align__(16) float As[2][BK][BN];
    const int n_rows = *e.n_rows;
    const int row0 = blockIdx.y * BM;
    if (row0 >= n_rows) return;
    int kbps, n_split;
    split_plan(e.sp, n_rows, &kbps, &n_split);
    const int split = blockIdx.z;
    if (split >= n_split) return;
    const DevProblem &pb = e.pb;
    const int nd = (int)pb.nd_pad;
    const int d0 = blockIdx.x * BN;
    const int n_beg = split * kbps * BK;
    const int n_end = min((int)pb.np_pad, n_beg + kbps * BK);
    const int tid = threadIdx.x;
    const int tr = tid >> 4, tc = tid & 15;

    const int lr = tid >> 2, lk = (tid & 3) * 4;           // G tile: row, point offset
    const bool row_ok = row0 + lr < n_rows;
    const float *Gp = e.G + (size_t)(row0 + lr) * pb.np_pad + lk;
    const int ak = tid >> 5, ac = (tid & 31) * 4;           // A tile: point, dwell offset
    const bool c_ok = d0 + ac < nd;
    const float *Ap = pb.A32 + (size_t)ak * nd + d0 + ac;

    float4 rG, rA0, rA1;
    auto gload = [&](int n0) {
        rG = row_ok ? *reinterpret_cast<const float4 *>(Gp + n0) : make_float4(0, 0, 0, 0);
        rA0 = c_ok ? *reinterpret_cast<const float4 *>(Ap + (size_t)n0 * nd)
                   : make_float4(0, 0, 0, 0);
        rA1 = c_ok ? *reinterpret_cast<const float4 *>(Ap + (size_t)(n0 + 8) * nd)
                   : make_float4(0, 0, 0, 0);
    };
    auto sstore = [&](int buf) {
        Gs[buf][lk + 0][lr] = rG.x; Gs[buf][lk + 1][lr] = rG.y;
        Gs[buf][lk + 2][lr] = rG.z; Gs[buf][lk + 3][lr] = rG.w;
        *reinterpret_cast<float4 *>(&As[buf][ak][ac]) = rA0;
        *reinterpret_cast<float4 *>(&As[buf][ak + 8][ac]) = rA1;
    };

    float acc[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = 0.0f;

    const int nk = (n_end - n_beg) / BK;
    if (nk > 0) {
        gload(n_beg);
        sstore(0);
    }
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) gload(n_beg + (kt + 1) * BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 gq = *reinterpret_cast<const float4 *>(&Gs[buf][k][tr * 4]);
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][tc * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][64 + tc * 4]);
            const float gv[4] = {gq.x, gq.y, gq.z, gq.w};
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(gv[r], av[c], acc[r][c]);
        }
        if (kt + 1 < nk) sstore(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int row = row0 + tr * 4 + r;
        if (row >= n_rows) continue;
        float *out = e.gpart + ((size_t)split * n_rows + row) * nd + d0;
        if (d0 + tc * 4 < nd)
            *reinterpret_cast<float4 *>(out + tc * 4) =
                make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
        if (d0 + 64 + tc * 4 < nd)
            *reinterpret_cast<float4 *>(out + 64 + tc * 4) =
                make_float4(acc[r][4], acc[r][5], acc[r][6], acc[r][7]);
    }
}

}  // namespace

int32_t simt_n_ptiles(const DevProblem &pb) { return (int32_t)(pb.np_pad / BN); }

SplitPlan simt_split_plan(const DevProblem &pb)
{
    SplitPlan p{};
    p.rows_per_tile = BM;
    p.other_tiles = (int32_t)ceil_div(pb.nd_pad, BN);
    p.kb_total = (int32_t)(pb.np_pad / BK);
    p.target_ctas = 148 * 2 * 2;     // two CTAs per SM, two waves
    p.max_split = (int32_t)std::min<int64_t>(148, p.kb_total);
    p.min_kb = 32;                   // splits of at least 512 points (see tc_split_plan)
    return p;
}

cudaError_t launch_gemm1_simt(const EvalArgs &e, int32_t mode, cudaStream_t st)
{
    const DevProblem &hpb = e.pb;
    dim3 grid((unsigned)(hpb.np_pad / BN), (unsigned)ceil_div(e.cap, BM));
    if (e.dT) k_gemm1<true><<<grid, NT, 0, st>>>(e, mode);
    else k_gemm1<false><<<grid, NT, 0, st>>>(e, mode);
    return cudaGetLastError();
}

cudaError_t launch_gemm2_simt(const EvalArgs &e, cudaStream_t st)
{
    const DevProblem &hpb = e.pb;
    dim3 grid((unsigned)ceil_div(hpb.nd_pad, BN), (unsigned)ceil_div(e.cap, BM),
              (unsigned)e.sp.max_split);
    k_gemm2<<<grid, NT, 0, st>>>(e);
    return cudaGetLastError();
}

}  // namespace gmco
