// Dose calculation points of the synthetic prostate geometry on the GPU: the sampling half of
// step (i) of the planning flow (Sec. 2.2.1; the clinical flow creates points from contours,
// which needs DICOM data that is not available, so the structures here are the analytic
// volumes of the workload: prostate ellipsoid, urethra and rectum cylinders, bladder sphere).
//
// Rule (restated by the test oracle, which reproduces it bit for bit):
//   candidate k of structure s has coordinates lo_a + u_a w_a (a = x, y, z) in the structure's
//   bounding box (corner lo, widths w), u_a = the top 24 bits of SplitMix64 output number
//   s 2^40 + 4 k + a, times 2^-24; point i of structure s is its i-th accepted candidate in
//   order of k.  Acceptance: prostate = inside the ellipsoid and not in the urethra; urethra =
//   inside its cylinder; rectum = inside its cylinder and not in the prostate; bladder =
//   inside its sphere and in neither the prostate nor the rectum.
// Every floating point step is a single IEEE FP32 operation, rounded to nearest (explicit _rn
// intrinsics, no contraction into FMA), in the order written, so that any IEEE FP32
// implementation of the rule takes the same decisions.
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

namespace gmco {
namespace {

struct Geo32 {
    float a, b, c, ru, rr, yr, hr, rb, zb;
};

__device__ __forceinline__ uint64_t splitmix64_pt(uint64_t seed, uint64_t n)
{
    // published SplitMix64 (Steele, Lea and Flood 2014): Weyl state seed + (n + 1) gamma,
    // then the variant-13 finaliser
    uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float sq(float v) { return __fmul_rn(v, v); }

__device__ __forceinline__ bool in_prostate(const Geo32 &g, float x, float y, float z)
{
    const float s = __fadd_rn(__fadd_rn(sq(__fdiv_rn(x, g.a)), sq(__fdiv_rn(y, g.b))), sq(__fdiv_rn(z, g.c)));
    return s <= 1.0f;
}
__device__ __forceinline__ bool in_urethra(const Geo32 &g, float x, float y, float z)
{
    return __fadd_rn(sq(x), sq(y)) <= sq(g.ru) && fabsf(z) <= g.c;
}
__device__ __forceinline__ bool in_rectum(const Geo32 &g, float x, float y, float z)
{
    return __fadd_rn(sq(x), sq(__fsub_rn(y, g.yr))) <= sq(g.rr) && fabsf(z) <= g.hr;
}
__device__ __forceinline__ bool in_bladder(const Geo32 &g, float x, float y, float z)
{
    return __fadd_rn(__fadd_rn(sq(x), sq(y)), sq(__fsub_rn(z, g.zb))) <= sq(g.rb);
}

// Candidate k of structure s: its coordinates and whether it is accepted.
__device__ __forceinline__ bool candidate(const Geo32 &g, int s, uint64_t seed, uint64_t k, float *p)
{
    float lo[3], w[3];
    if (s == 0) {
        lo[0] = -g.a; lo[1] = -g.b; lo[2] = -g.c;
        w[0] = __fadd_rn(g.a, g.a); w[1] = __fadd_rn(g.b, g.b); w[2] = __fadd_rn(g.c, g.c);
    } else if (s == 1) {
        lo[0] = -g.ru; lo[1] = -g.ru; lo[2] = -g.c;
        w[0] = __fadd_rn(g.ru, g.ru); w[1] = w[0]; w[2] = __fadd_rn(g.c, g.c);
    } else if (s == 2) {
        lo[0] = -g.rr; lo[1] = __fsub_rn(g.yr, g.rr); lo[2] = -g.hr;
        w[0] = __fadd_rn(g.rr, g.rr); w[1] = w[0]; w[2] = __fadd_rn(g.hr, g.hr);
    } else {
        lo[0] = -g.rb; lo[1] = -g.rb; lo[2] = __fsub_rn(g.zb, g.rb);
        w[0] = __fadd_rn(g.rb, g.rb); w[1] = w[0]; w[2] = w[0];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const uint64_t z = splitmix64_pt(seed, ((uint64_t)s << 40) + 4ull * k + (uint64_t)a);
        const float u = (float)(uint32_t)(z >> 40) * 0x1p-24f;   // exact: 24-bit integer
        p[a] = __fadd_rn(lo[a], __fmul_rn(u, w[a]));
    }
    const float x = p[0], y = p[1], z = p[2];
    if (s == 0) return in_prostate(g, x, y, z) && !in_urethra(g, x, y, z);
    if (s == 1) return in_urethra(g, x, y, z);
    if (s == 2) return in_rectum(g, x, y, z) && !in_prostate(g, x, y, z);
    return in_bladder(g, x, y, z) && !in_prostate(g, x, y, z) && !in_rectum(g, x, y, z);
}

constexpr int kPtBlock = 256;

// Accepted candidates per block of 256 candidates.
__global__ void __launch_bounds__(kPtBlock) k_pt_count(Geo32 g, int32_t s, uint64_t seed, int64_t K,
                                                      int32_t *__restrict__ counts)
{
    const int64_t k = (int64_t)blockIdx.x * kPtBlock + threadIdx.x;
    float p[3];
    const bool acc = k < K && candidate(g, s, seed, (uint64_t)k, p);
    const int n = __syncthreads_count(acc ? 1 : 0);
    if (threadIdx.x == 0) counts[blockIdx.x] = n;
}

// Writes the accepted candidates of each block at their ranks (offset of the block + rank in
// the block), the first n of the structure only.
__global__ void __launch_bounds__(kPtBlock) k_pt_write(Geo32 g, int32_t s, uint64_t seed, int64_t K,
                                                      const int64_t *__restrict__ offsets, int64_t n,
                                                      float *__restrict__ pts, int32_t *__restrict__ sid)
{
    __shared__ int32_t warp_n[kPtBlock / 32];
    const int64_t k = (int64_t)blockIdx.x * kPtBlock + threadIdx.x;
    float p[3];
    const bool acc = k < K && candidate(g, s, seed, (uint64_t)k, p);
    const unsigned ball = __ballot_sync(0xffffffffu, acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_n[warp] = __popc(ball);
    __syncthreads();
    int before = 0;
    for (int w2 = 0; w2 < warp; ++w2) before += warp_n[w2];
    const int64_t rank = offsets[blockIdx.x] + before + __popc(ball & ((1u << lane) - 1u));
    if (acc && rank < n) {
        pts[rank * 3 + 0] = p[0];
        pts[rank * 3 + 1] = p[1];
        pts[rank * 3 + 2] = p[2];
        sid[rank] = s;
    }
}

}  // namespace

cudaError_t sample_points_dev(const double *geo, const int64_t *counts, uint64_t seed, float *pts,
                              int32_t *sid, cudaStream_t st, int32_t *short_struct)
{
    const Geo32 g{(float)geo[0], (float)geo[1], (float)geo[2], (float)geo[3], (float)geo[4],
                  (float)geo[5], (float)geo[6], (float)geo[7], (float)geo[8]};
    *short_struct = -1;
    int64_t base = 0;
    int32_t *d_counts = nullptr;
    int64_t *d_off = nullptr;
    int64_t cap_blocks = 0;
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < 4 && e == cudaSuccess; ++s) {
        const int64_t n = counts[s];
        if (n == 0) continue;
        // enough candidates for the lowest acceptance of these shapes (about 0.5), doubled
        // while short
        int64_t K = 3 * n + 1024, total = 0;
        std::vector<int32_t> hc;
        int64_t nb = 0;
        for (int round = 0; round < 8; ++round, K *= 2) {
            nb = (K + kPtBlock - 1) / kPtBlock;
            if (nb > 0x7fffffffLL) break;   // beyond one launch's grid: treated as short
            if (nb > cap_blocks) {
                cudaFree(d_counts);
                cudaFree(d_off);
                d_counts = nullptr;
                d_off = nullptr;
                if ((e = cudaMalloc(&d_counts, nb * sizeof(int32_t))) != cudaSuccess) break;
                if ((e = cudaMalloc(&d_off, nb * sizeof(int64_t))) != cudaSuccess) break;
                cap_blocks = nb;
            }
            k_pt_count<<<(unsigned)nb, kPtBlock, 0, st>>>(g, s, seed, K, d_counts);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            hc.resize((size_t)nb);
            if ((e = cudaMemcpyAsync(hc.data(), d_counts, nb * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                     st)) != cudaSuccess)
                break;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
            total = 0;
            for (int32_t c : hc) total += c;
            if (total >= n) break;
        }
        if (e != cudaSuccess) break;
        if (total < n) {
            *short_struct = s;
            break;
        }
        std::vector<int64_t> off((size_t)nb);
        int64_t acc = 0;
        for (int64_t b = 0; b < nb; ++b) {
            off[(size_t)b] = acc;
            acc += hc[(size_t)b];
        }
        if ((e = cudaMemcpyAsync(d_off, off.data(), nb * sizeof(int64_t), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
            break;
        k_pt_write<<<(unsigned)nb, kPtBlock, 0, st>>>(g, s, seed, K, d_off, n, pts + base * 3, sid + base);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;   // off lives on the host
        base += n;
    }
    cudaFree(d_counts);
    cudaFree(d_off);
    return e;
}

}  // namespace gmco
