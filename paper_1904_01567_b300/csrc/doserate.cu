// Dose rate matrix calculation, step (i) of the GPU planning flow (Sec. 2.2.1: one value per
// dose calculation point and dwell position), feeding Eq. (dose).  The paper does not state its
// dose-rate model; this is the isotropic point source
//   A_il = K g(r) / r^2,   r = max(|p_i - q_l|, r_min),   g(r) = g0 + g1 r + g2 r^2,
// with K = Lambda S_K times a unit factor, evaluated in FP32 (1 / r by rsqrtf) and written
// row-major (points x dwells), the layout gmco_create_problem takes.  The HBM write of A
// (4 bytes per element) bounds the kernel.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"

namespace gmco {

namespace {

constexpr int kRateThreads = 256;
constexpr int kRateMaxDwell = 1024;   // dwell coordinates staged in shared memory
constexpr int kRateRows = 32;         // point rows whose coordinates one load brings in

// Blocks take 32 point rows at a time (their coordinates staged in shared memory by one
// coalesced load, so that no row waits on its own load); the block's threads cover
// consecutive dwells of each row (coalesced stores).  The dwell coordinates sit in shared
// memory for the whole launch.
__global__ void __launch_bounds__(kRateThreads)
k_dose_rate(const float *__restrict__ pts, int64_t n_pnt, const float *__restrict__ dw, int32_t n_dwell,
            float K, float r_min, float r_min2, float rinv_min, float g0, float g1, float g2,
            float *__restrict__ A, int32_t *bad)
{
    __shared__ float s_dw[3][kRateMaxDwell];
    for (int l = threadIdx.x; l < n_dwell; l += blockDim.x) {
        s_dw[0][l] = dw[3 * (size_t)l];
        s_dw[1][l] = dw[3 * (size_t)l + 1];
        s_dw[2][l] = dw[3 * (size_t)l + 2];
    }
    __shared__ float s_pt[kRateRows * 3];
    __syncthreads();
    bool neg = false;
    for (int64_t i0 = (int64_t)blockIdx.x * kRateRows; i0 < n_pnt; i0 += (int64_t)gridDim.x * kRateRows) {
        const int rows = (int)min((int64_t)kRateRows, n_pnt - i0);
        if ((int)threadIdx.x < 3 * rows) s_pt[threadIdx.x] = pts[3 * i0 + threadIdx.x];
        __syncthreads();
        for (int rr = 0; rr < rows; ++rr) {
            const float px = s_pt[3 * rr], py = s_pt[3 * rr + 1], pz = s_pt[3 * rr + 2];
            float *row = A + (i0 + rr) * n_dwell;
            for (int l = threadIdx.x; l < n_dwell; l += blockDim.x) {
                const float dx = px - s_dw[0][l], dy = py - s_dw[1][l], dz = pz - s_dw[2][l];
                const float r2 = dx * dx + dy * dy + dz * dz;
                // 1 / r from one reciprocal square root (no square root and division sequences);
                // a NaN distance stays NaN (the compare is false) and is caught below
                const bool clamp = r2 < r_min2;
                const float rinv = clamp ? rinv_min : rsqrtf(r2);
                const float r = clamp ? r_min : r2 * rinv;
                const float g = (g2 * r + g1) * r + g0;
                neg = neg || !(g > 0.0f);
                row[l] = K * g * (rinv * rinv);
            }
        }
        __syncthreads();   // the next rows' coordinates overwrite s_pt
    }
    if (neg) atomicOr(bad, 1);
}

}  // namespace

cudaError_t launch_dose_rate(const float *pts, int64_t n_pnt, const float *dw, int32_t n_dwell,
                             const double *src, float *A, int32_t *bad, cudaStream_t st)
{
    if (n_dwell < 1 || n_dwell > kRateMaxDwell || n_pnt < 1) return cudaErrorInvalidValue;
    // src: Lambda, S_K, unit factor, r_min, g0, g1, g2
    const float K = (float)(src[0] * src[1] * src[2]);
    const int64_t chunks = (n_pnt + kRateRows - 1) / kRateRows;
    const int64_t blocks = chunks < 148 * 8 ? chunks : 148 * 8;
    const float r_min = (float)src[3];
    k_dose_rate<<<(unsigned)blocks, kRateThreads, 0, st>>>(pts, n_pnt, dw, n_dwell, K, r_min, r_min * r_min,
                                                          1.0f / r_min, (float)src[4], (float)src[5],
                                                          (float)src[6], A, bad);
    return cudaGetLastError();
}

}  // namespace gmco
