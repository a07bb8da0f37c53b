// Plan-pool post-processing of gMCO: the RTOG / RTOG+ evaluation of each plan (Sec. 2.3.1), the
// selection of one plan from the pool (Sec. 2.4) and the non-dominated filter of Sec. 2.2.4.
// Small kernels over per-plan values; every decision is taken in FP64 from the same inputs as
// the oracle, so classes, the selected index and the non-dominated flags are exact.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"

namespace gmco {

namespace {

constexpr int kPoolThreads = 1024;

// Class of one plan from its DVH row (V100 %, D90 %, urethra D10 %, rectum V75 %, bladder V75 %)
// and the criteria c = {V100 min (RTOG), V100 min (RTOG+), D10 max, V75 max cc, rectum cc,
// bladder cc}: 2 = RTOG+, 1 = RTOG, 0 = invalid.  Also whether target and urethra pass and the
// two V75 volumes' sum (cc), the invalid plans' ranking.
struct PlanEval {
    int cls;
    bool tu_ok;
    double v100, oar_cc;
};

__device__ __forceinline__ PlanEval eval_plan(const float *row, const double *c)
{
    PlanEval e;
    e.v100 = (double)row[0];
    const double d10 = (double)row[2];
    const double rect_cc = (double)row[3] * c[4] / 100.0, blad_cc = (double)row[4] * c[5] / 100.0;
    const bool target = e.v100 >= c[0], urethra = d10 < c[2];
    const bool oars = rect_cc < c[3] && blad_cc < c[3];
    e.tu_ok = target && urethra;
    e.oar_cc = rect_cc + blad_cc;
    e.cls = (target && urethra && oars) ? (e.v100 >= c[1] ? 2 : 1) : 0;
    return e;
}

// Whether plan a ranks above plan b (indices ia < ib break ties): higher class; among valid
// plans higher V100; among invalid ones, passing target and urethra, then the lower V75 sum.
__device__ __forceinline__ bool better(const PlanEval &a, int ia, const PlanEval &b, int ib)
{
    if (a.cls != b.cls) return a.cls > b.cls;
    if (a.cls > 0) {
        if (a.v100 != b.v100) return a.v100 > b.v100;
    } else {
        if (a.tu_ok != b.tu_ok) return a.tu_ok;
        if (a.oar_cc != b.oar_cc) return a.oar_cc < b.oar_cc;
    }
    return ia < ib;
}

// One block: classes of every plan, then the best plan by a fixed-order tree reduction (the
// order of the comparisons does not matter: `better` is a strict total order).
__global__ void __launch_bounds__(kPoolThreads)
k_rtog(const float *__restrict__ dvh, int64_t P, const double *__restrict__ crit, int32_t *__restrict__ cls,
       int32_t *__restrict__ selected)
{
    __shared__ double c[6];
    __shared__ int32_t s_idx[kPoolThreads];
    if (threadIdx.x < 6) c[threadIdx.x] = crit[threadIdx.x];
    __syncthreads();
    int best = -1;
    PlanEval be{};
    for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
        const PlanEval e = eval_plan(dvh + i * GMCO_DVH_K, c);
        cls[i] = e.cls;
        if (best < 0 || better(e, (int)i, be, best)) {
            best = (int)i;
            be = e;
        }
    }
    s_idx[threadIdx.x] = best;
    __syncthreads();
    for (int w = kPoolThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const int a = s_idx[threadIdx.x], b = s_idx[threadIdx.x + w];
            if (b >= 0 && (a < 0 || better(eval_plan(dvh + (int64_t)b * GMCO_DVH_K, c), b,
                                            eval_plan(dvh + (int64_t)a * GMCO_DVH_K, c), a)))
                s_idx[threadIdx.x] = b;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *selected = s_idx[0];
}

// Plan i is dominated when another plan is no worse in every objective and better in one
// (all objectives minimised).  One thread per plan, the other plans' rows read in tiles of
// shared memory.
constexpr int kParetoTile = 256, kParetoMaxK = 16;

__global__ void __launch_bounds__(kParetoTile)
k_pareto(const double *__restrict__ obj, int64_t P, int32_t K, int32_t *__restrict__ nondom)
{
    __shared__ double tile[kParetoTile * kParetoMaxK];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double mine[kParetoMaxK];
#pragma unroll
    for (int k = 0; k < kParetoMaxK; ++k) mine[k] = (i < P && k < K) ? obj[i * K + k] : 0.0;
    bool dominated = false;
    for (int64_t j0 = 0; j0 < P; j0 += kParetoTile) {
        const int n = (int)min((int64_t)kParetoTile, P - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < n * K; t += blockDim.x) tile[t] = obj[j0 * K + t];
        __syncthreads();
        if (i < P && !dominated) {
            for (int jj = 0; jj < n; ++jj) {
                bool le = true, lt = false;
#pragma unroll
                for (int k = 0; k < kParetoMaxK; ++k) {
                    if (k < K) {
                        const double o = tile[jj * K + k];
                        le = le && o <= mine[k];
                        lt = lt || o < mine[k];
                    }
                }
                if (le && lt) {
                    dominated = true;
                    break;
                }
            }
        }
    }
    if (i < P) nondom[i] = dominated ? 0 : 1;
}

}  // namespace

cudaError_t launch_rtog(const float *dvh, int64_t P, const double *crit, int32_t *cls, int32_t *selected,
                        cudaStream_t st)
{
    if (P < 1 || P > (int64_t)1 << 30) return cudaErrorInvalidValue;
    k_rtog<<<1, kPoolThreads, 0, st>>>(dvh, P, crit, cls, selected);
    return cudaGetLastError();
}

cudaError_t launch_pareto(const double *obj, int64_t P, int32_t K, int32_t *nondom, cudaStream_t st)
{
    if (P < 1 || K < 1 || K > kParetoMaxK) return cudaErrorInvalidValue;
    const int64_t blocks = (P + kParetoTile - 1) / kParetoTile;
    k_pareto<<<(unsigned)blocks, kParetoTile, 0, st>>>(obj, P, K, nondom);
    return cudaGetLastError();
}

}  // namespace gmco
