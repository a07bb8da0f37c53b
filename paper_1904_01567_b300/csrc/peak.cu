// Measurement aid: the FP32 fused multiply-add throughput of the device, the pipe peak against
// which the FP32 form's SIMT contractions are reported.  Every thread runs 16 independent FMA
// chains (enough to cover the FMA latency at full occupancy); the chains' results are combined
// and stored so that no FMA is dead code.  Two kernels: scalar FFMA, and the paired FP32 form
// (two lanes of a 64-bit register per instruction), which doubles the FP32 rate on sm_100-class
// devices where it is supported.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace gmco {
namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(256) k_ffma(float *out, int32_t iters, float a, float b)
{
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_ffma2(float *out, int32_t iters, float a, float b)
{
    float2 v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)c * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = __ffma2_rn(v[c], a2, b2);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c].x + v[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace gmco

extern "C" {

// tflops[0]: scalar FFMA, tflops[1]: paired FP32 FMA, each the best of `reps` timed launches
// (CUDA events, after one warm-up) of 8 resident blocks of 256 threads per SM running `iters`
// iterations of 16 FMA chains.  Synchronous; allocates one small device buffer.
gmco_status gmco_fp32_peak(int32_t iters, int32_t reps, double *tflops)
{
    using namespace gmco;
    if (iters < 1 || reps < 1 || !tflops) return GMCO_EINVAL;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return GMCO_ECUDA;
    }
    const int blocks = n_sm * 8, threads = 256;
    float *out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return GMCO_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    gmco_status st = GMCO_OK;
    for (int kind = 0; kind < 2 && st == GMCO_OK; ++kind) {
        double best = 0.0;
        for (int r = 0; r < reps + 1; ++r) {
            cudaEventRecord(e0);
            if (kind == 0) k_ffma<<<blocks, threads>>>(out, iters, 0.999f, 1e-3f);
            else k_ffma2<<<blocks, threads>>>(out, iters, 0.999f, 1e-3f);
            cudaEventRecord(e1);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
                st = GMCO_ECUDA;
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double flop = 2.0 * (kind == 0 ? 1.0 : 2.0) * kChains * (double)iters * blocks * threads;
            if (r > 0) best = std::max(best, flop / (ms * 1e-3) / 1e12);
        }
        tflops[kind] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return st;
}

}  // extern "C"
