// DVH indices of Sec. 2.3.1 from per-point doses, one CTA per plan:
//   V100 (structure 0), D90 (structure 0), D10 (structure 1), V75 (structures 2 and 3).
// V_x counts points with d >= x % of Rx; D_x is the k-th largest dose of the structure with
// k = ceil(x/100 N) (the lowest dose received by the hottest x % of its points), found by an
// exact 4-pass radix select on order-preserving 32-bit keys of the FP32 doses.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"

namespace gmco {

namespace {

__device__ __forceinline__ uint32_t order_key(float d)
{
    const uint32_t b = __float_as_uint(d);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float key_value(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// k-th largest dose (1-based) among points of structure s; all threads return it.
__device__ float kth_largest(const float *__restrict__ d, const int8_t *__restrict__ sid,
                             int64_t n, int s, int64_t k, uint32_t *hist, uint32_t *bcast)
{
    uint32_t prefix = 0, mask = 0;
    int64_t krem = k;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            if (sid[i] != s) continue;
            const uint32_t key = order_key(d[i]);
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t cum = 0;
            int sel = 0;
            for (int b = 255; b >= 0; --b) {
                if (cum + (int64_t)hist[b] >= krem) { sel = b; break; }
                cum += hist[b];
            }
            bcast[0] = (uint32_t)sel;
            bcast[1] = (uint32_t)(krem - cum);
        }
        __syncthreads();
        prefix |= bcast[0] << shift;
        mask |= 255u << shift;
        krem = bcast[1];
        __syncthreads();
    }
    return key_value(prefix);
}

__global__ void k_dvh(const float *__restrict__ D, int64_t ld, const int8_t *__restrict__ sid,
                      int64_t n, int32_t n_struct, const int32_t *__restrict__ rows,
                      int32_t P, double rx, float *__restrict__ out)
{
    __shared__ uint32_t hist[256];
    __shared__ uint32_t bcast[2];
    __shared__ unsigned long long cnt[7];
    const int r = blockIdx.x;
    if (r >= P) return;
    const int plan = rows ? rows[r] : r;
    const float *d = D + (size_t)r * ld;
    if (threadIdx.x < 7) cnt[threadIdx.x] = 0;
    __syncthreads();
    const float t100 = (float)rx, t75 = (float)(0.75 * rx);
    unsigned long long c[7] = {0, 0, 0, 0, 0, 0, 0};  // N0..N3, V100, V75(2), V75(3)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int s = sid[i];
        const float v = d[i];
        if (s >= 0 && s < 4) c[s]++;
        if (s == 0 && v >= t100) c[4]++;
        if (s == 2 && v >= t75) c[5]++;
        if (s == 3 && v >= t75) c[6]++;
    }
    for (int q = 0; q < 7; ++q)
        if (c[q]) atomicAdd(&cnt[q], c[q]);
    __syncthreads();
    const int64_t N0 = (int64_t)cnt[0], N1 = (int64_t)cnt[1], N2 = (int64_t)cnt[2],
                  N3 = (int64_t)cnt[3];
    float res[GMCO_DVH_K];
    for (int q = 0; q < GMCO_DVH_K; ++q) res[q] = __int_as_float(0x7fc00000);  // NaN
    if (n_struct > 0 && N0 > 0) {
        res[0] = (float)(100.0 * (double)cnt[4] / (double)N0);
        const float d90 = kth_largest(d, sid, n, 0, (9 * N0 + 9) / 10, hist, bcast);
        res[1] = (float)(100.0 * (double)d90 / rx);
    }
    if (n_struct > 1 && N1 > 0) {
        const float d10 = kth_largest(d, sid, n, 1, (N1 + 9) / 10, hist, bcast);
        res[2] = (float)(100.0 * (double)d10 / rx);
    }
    if (n_struct > 2 && N2 > 0) res[3] = (float)(100.0 * (double)cnt[5] / (double)N2);
    if (n_struct > 3 && N3 > 0) res[4] = (float)(100.0 * (double)cnt[6] / (double)N3);
    if (threadIdx.x == 0)
        for (int q = 0; q < GMCO_DVH_K; ++q) out[(size_t)plan * GMCO_DVH_K + q] = res[q];
}

}  // namespace

cudaError_t launch_dvh(const DevProblem &pb, const float *D, int64_t ld, const int32_t *rows,
                       int32_t P, double rx, float *dvh_out, cudaStream_t st)
{
    if (P <= 0) return cudaSuccess;
    k_dvh<<<P, 256, 0, st>>>(D, ld, pb.sid, pb.n_pnt, pb.n_struct, rows, P, rx, dvh_out);
    return cudaGetLastError();
}

}  // namespace gmco
