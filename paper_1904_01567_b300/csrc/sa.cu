// The stochastic engine gSA of Sec. 2.2.1: steps (ii)-(v) repeated for every plan at once.  Each
// iteration moves all dwell weights of every plan (step (ii), k_sa_propose), evaluates the moved
// plans with the library's dose GEMM and penalty epilogue (steps (iii)-(v), the same kernels as
// the quasi-Newton engine's evaluation), and keeps or drops each plan's move by the Metropolis
// rule (k_sa_accept).  The paper gives neither the move nor the cooling schedule; the ones here:
//   x'_l = x_l + delta_k (2 u - 1) for every dwell l (t = x^2 stays non-negative, Sec. 2.1.2),
//   accept when F(x') - F(x) <= -T_k F(x_0) ln v,
// with u, v uniform draws and delta_k, T_k passed in by the host.  Draws are SplitMix64 outputs
// (Steele, Lea and Flood 2014) at a counter of (plan, iteration, dwell), so an engine that draws
// the same counters sees the same numbers whatever its launch shape.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"

namespace gmco {

namespace {

constexpr int kSaThreads = 128;
constexpr uint64_t kAcceptDraw = (1u << 21) - 1;   // the dwell slot of a plan's acceptance draw

// Output n (0-based) of SplitMix64 seeded with `seed`: the Weyl state seed + (n + 1) gamma
// through the generator's finaliser.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Counter of the draw of plan p, iteration k, dwell l: k in bits 42.., p in 21..41, l in 0..20.
__device__ __forceinline__ uint64_t draw_counter(int64_t p, int32_t k, uint64_t l)
{
    return ((uint64_t)k << 42) | ((uint64_t)p << 21) | l;
}

// Moved weights of plan j (one block per plan): x = xc + delta (2 u - 1), u the top 53 bits of
// the draw times 2^-53.  The step is formed in FP64 and rounded once to the FP32 weights.
__global__ void __launch_bounds__(kSaThreads)
k_sa_propose(float *__restrict__ x, const float *__restrict__ xc, int64_t nd, int64_t nd_pad,
             uint64_t seed, int32_t k, double delta)
{
    const int64_t j = blockIdx.x;
    for (int64_t l = threadIdx.x; l < nd; l += blockDim.x) {
        const uint64_t z = splitmix64(seed, draw_counter(j, k, (uint64_t)l));
        const double r = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
        x[j * nd_pad + l] = xc[j * nd_pad + l] + (float)(delta * r);
    }
}

// Metropolis decision of plan j on its evaluated move (objective Ft[j]), in FP64; then the moved
// weights become the current ones (accepted) and the best ones (a new lowest objective).
// k < 0: the first evaluation, at the start point, which sets the current, best and initial
// objectives.  A non-finite objective never passes the test.
__global__ void __launch_bounds__(kSaThreads)
k_sa_accept(const float *__restrict__ x, float *__restrict__ xc, float *__restrict__ xb,
            int64_t nd_pad, const double *__restrict__ Ft, double *__restrict__ Fc,
            double *__restrict__ Fb, double *__restrict__ F0, int32_t *__restrict__ acc,
            uint64_t seed, int32_t k, double temp)
{
    const int64_t j = blockIdx.x;
    __shared__ int s_copy;   // bit 0: to the current weights, bit 1: to the best weights
    if (threadIdx.x == 0) {
        const double f = Ft[j];
        int copy = 0;
        if (k < 0) {
            F0[j] = f;
            Fc[j] = f;
            Fb[j] = f;
            acc[j] = 0;
            copy = 3;
        } else {
            const uint64_t z = splitmix64(seed, draw_counter(j, k, kAcceptDraw));
            const double v = ((double)(z >> 11) + 1.0) * 0x1.0p-53;   // (0, 1]
            const double theta = -temp * F0[j] * log(v);
            if (f - Fc[j] <= theta) {
                Fc[j] = f;
                acc[j] += 1;
                copy = 1;
                if (f < Fb[j]) {
                    Fb[j] = f;
                    copy = 3;
                }
            }
        }
        s_copy = copy;
    }
    __syncthreads();
    const int copy = s_copy;
    if (!copy) return;
    for (int64_t l = threadIdx.x; l < nd_pad; l += blockDim.x) {
        const float v = x[j * nd_pad + l];
        if (copy & 1) xc[j * nd_pad + l] = v;
        if (copy & 2) xb[j * nd_pad + l] = v;
    }
}

}  // namespace

cudaError_t launch_sa_propose(float *x, const float *xc, int64_t P, int64_t nd, int64_t nd_pad,
                              uint64_t seed, int32_t k, double delta, cudaStream_t st)
{
    if (P < 1 || nd < 1 || nd >= (int64_t)kAcceptDraw || k < 0) return cudaErrorInvalidValue;
    k_sa_propose<<<(unsigned)P, kSaThreads, 0, st>>>(x, xc, nd, nd_pad, seed, k, delta);
    return cudaGetLastError();
}

cudaError_t launch_sa_accept(const float *x, float *xc, float *xb, int64_t P, int64_t nd_pad,
                             const double *Ft, double *Fc, double *Fb, double *F0, int32_t *acc,
                             uint64_t seed, int32_t k, double temp, cudaStream_t st)
{
    if (P < 1) return cudaErrorInvalidValue;
    k_sa_accept<<<(unsigned)P, kSaThreads, 0, st>>>(x, xc, xb, nd_pad, Ft, Fc, Fb, F0, acc, seed, k,
                                                    temp);
    return cudaGetLastError();
}

}  // namespace gmco
