// Learned warm start: a per-dwell-position multilayer perceptron that maps 10 geometric
// features of a dwell position and the 4 penalty weights of a plan to a dwell time,
//     x0 = [f_1..f_10, log10 max(w_1, 1e-3) .. log10 max(w_4, 1e-3)]      (14 inputs)
//     h_l = GELU(h_{l-1} W_l + b_l), l = 1, 2, 3 (width 128, GELU(z) = z Phi(z) with erf)
//     t = softplus(h_3 . w_4 + b_4)  (seconds), floored by the caller's t_floor.
// Trained on converged plans with the mean squared error of t and Adam; BF16 weights and
// activations in the products, FP32 accumulation, FP32 master weights.  The paper has no
// learned component: this is the warm-start extension of its batched solve.
//
// Kernels:
//   k_mlp_infer_tc          inference on the fifth-generation tensor cores: tcgen05.mma with
//                           the weights copied into shared memory by the TMA unit, FP32
//                           accumulators in TMEM, bias + GELU epilogues that write the next
//                           layer's BF16 operand; persistent grid, three 128-row tiles in
//                           flight per CTA
//   k_mlp_train             training forward and backward of 16-row tiles per warp on
//                           warp-level BF16 MMA (m16n8k16, FP32 accumulators in registers):
//                           activations carried from one layer's accumulators to the next
//                           layer's operand fragments in registers, weights in shared memory;
//                           the loss and the backward pass of each tile in registers
//                           (dz_3 -> dh_2 -> dz_2 -> dh_1 -> dz_1 with the transposed products
//                           h W^T); writes the layer inputs H_{l-1} and the pre-activation
//                           gradients dZ_l feature-major for the weight gradients, and per-CTA
//                           partial sums of the bias gradients
//   k_mlp_dw                dW_l = H_{l-1}^T dZ_l, split over row ranges, per-CTA partials
//   k_mlp_reduce            fixed-order sums of the per-CTA partials into the gradient
//   k_mlp_adam              Adam on the FP32 master weights, then the BF16 copies
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "gmco.h"
#include "tcgen05.cuh"

namespace {

constexpr int NIN = 14, NFEAT = 10, NW = 4, KIN = 16, HID = 128;
constexpr int WARPS = 8, ROWS_W = 16, ROWS_CTA = WARPS * ROWS_W;
constexpr int LDH = HID + 8;   // padded row (bf16) of the 128-wide weight copies in smem
constexpr int LD1 = KIN + 8;   // padded row of W1^T
// flat FP32 parameter layout (the C ABI's): W1 [14][128], b1, W2 [128][128], b2, W3, b3, w4, b4
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NIN * HID, OFF_W2 = OFF_B1 + HID,
              OFF_B2 = OFF_W2 + HID * HID, OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID * HID,
              OFF_W4 = OFF_B3 + HID, OFF_B4 = OFF_W4 + HID, NPARAM = OFF_B4 + 1;
static_assert(NPARAM == GMCO_MLP_NPARAM, "parameter count");
constexpr int NPART = 1 + 4 * HID + 1;   // per-CTA partials: loss, db1, db2, db3, dw4, db4
constexpr int MAX_CTAS = 148;

// BF16 weights as the kernels read them.
struct DevWeights {
    __nv_bfloat16 *Wt1;        // [128][16]  W1^T (n, k), k padded to 16 with zeros
    __nv_bfloat16 *Wt2, *Wt3;  // [128][128] W^T (n, k): forward operand
    __nv_bfloat16 *W2, *W3;    // [128][128] W (k, n): backward operand
    float *bias;               // b1, b2, b3, w4 (4 x 128) and b4
    uint8_t *img;              // shared-memory image of W1^T, W2^T, W3^T for k_mlp_infer_tc
};

// Rows of one call: dense (row = plan * n_dwell + dwell) or listed (pairs[row] = (feature
// row, weight row)).
struct RowSrc {
    const float *feat;      // [n_feat][10]
    const float *w;         // [n_w][4] raw penalty weights
    const int32_t *pairs;   // [R][2] or null (dense)
    int64_t n_dwell;        // dense mode
    int64_t R;
    const float *target;    // [R] (training)
};

struct TrainOut {
    __nv_bfloat16 *H0, *H1, *H2;      // [16][Rp], [128][Rp], [128][Rp]  layer inputs
    __nv_bfloat16 *dZ1, *dZ2, *dZ3;   // [128][Rp]                      pre-activation grads
    int64_t Rp;                       // row stride (R rounded up to 128)
    float *part;                      // [gridDim][NPART]
    float inv_R;                      // 1 / R (mean squared error)
};

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float2 unpack_bf16(uint32_t v)
{
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&v);
    return __bfloat1622float2(b);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_d(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
           z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ float softplus(float o) { return o > 20.0f ? o : log1pf(expf(o)); }
__device__ __forceinline__ float sigmoid(float o) { return 1.0f / (1.0f + expf(-o)); }

// Input column c of row r (0 past the row count and in the two padding columns).
__device__ __forceinline__ float in_val(const RowSrc &s, int64_t r, int c)
{
    if (r >= s.R || c >= NIN) return 0.0f;
    int64_t fr, wr;
    if (s.pairs) {
        fr = s.pairs[2 * r];
        wr = s.pairs[2 * r + 1];
    } else {
        fr = r % s.n_dwell;
        wr = r / s.n_dwell;
    }
    if (c < NFEAT) return s.feat[fr * NFEAT + c];
    return log10f(fmaxf(s.w[wr * NW + (c - NFEAT)], 1e-3f));
}

// acc (16 rows x 128 columns, C fragments of 16 n-tiles) -> operand fragments of 8 k-steps.
__device__ __forceinline__ void to_frag(const float (&acc)[16][4], uint32_t (&a)[8][4])
{
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        a[s][0] = pack_bf16(acc[2 * s][0], acc[2 * s][1]);
        a[s][1] = pack_bf16(acc[2 * s][2], acc[2 * s][3]);
        a[s][2] = pack_bf16(acc[2 * s + 1][0], acc[2 * s + 1][1]);
        a[s][3] = pack_bf16(acc[2 * s + 1][2], acc[2 * s + 1][3]);
    }
}

// acc += A (16 x 128, fragments) * B, B[k][n] read from smem rows of a (n, k)-major copy
// (forward: W^T) or a (k, n)-major one (backward: W, giving A W^T).
__device__ __forceinline__ void gemm_128(float (&acc)[16][4], const uint32_t (&a)[8][4],
                                         const __nv_bfloat16 *sB, int g, int t)
{
#pragma unroll
    for (int s = 0; s < 8; ++s) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const __nv_bfloat16 *row = sB + (size_t)(8 * j + g) * LDH + 16 * s + 2 * t;
            const uint32_t b0 = *reinterpret_cast<const uint32_t *>(row);
            const uint32_t b1 = *reinterpret_cast<const uint32_t *>(row + 8);
            mma16816(acc[j], a[s], b0, b1);
        }
    }
}

// Feature-major store of a 16 x 128 fragment set: out[col][row0 + row].
__device__ __forceinline__ void store_t(__nv_bfloat16 *out, int64_t ld, int64_t row0,
                                        const float (&v)[16][4], int g, int t)
{
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int c = 8 * j + 2 * t;
        out[(size_t)c * ld + row0 + g] = __float2bfloat16_rn(v[j][0]);
        out[(size_t)(c + 1) * ld + row0 + g] = __float2bfloat16_rn(v[j][1]);
        out[(size_t)c * ld + row0 + g + 8] = __float2bfloat16_rn(v[j][2]);
        out[(size_t)(c + 1) * ld + row0 + g + 8] = __float2bfloat16_rn(v[j][3]);
    }
}

// Column sums over the warp's 16 rows of a fragment set, added to sum[128] (lanes g = 0).
__device__ __forceinline__ void col_sums(const float (&v)[16][4], float *sum, int g, int t)
{
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        float s0 = v[j][0] + v[j][2], s1 = v[j][1] + v[j][3];
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (g == 0) {
            sum[8 * j + 2 * t] += s0;
            sum[8 * j + 2 * t + 1] += s1;
        }
    }
}

__global__ void __launch_bounds__(WARPS * 32, 1) k_mlp_train(DevWeights wt, RowSrc src, TrainOut tr)
{
    extern __shared__ __align__(16) uint8_t sm[];
    __nv_bfloat16 *sWt1 = reinterpret_cast<__nv_bfloat16 *>(sm);       // [128][LD1]
    __nv_bfloat16 *sWt2 = sWt1 + HID * LD1;                              // [128][LDH]
    __nv_bfloat16 *sWt3 = sWt2 + HID * LDH;
    __nv_bfloat16 *sW2 = sWt3 + HID * LDH;                               // backward operands
    __nv_bfloat16 *sW3 = sW2 + HID * LDH;
    __nv_bfloat16 *sZ = sW3 + HID * LDH;                                 // [2][8][16][128]
    __shared__ float sb[4 * HID + 1];
    __shared__ float sacc[WARPS][4 * HID + 2];   // per warp db1, db2, db3, dw4, db4, loss

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    for (int i = tid; i < HID * KIN; i += blockDim.x) sWt1[(i / KIN) * LD1 + i % KIN] = wt.Wt1[i];
    for (int i = tid; i < HID * HID; i += blockDim.x) {
        const int r = i / HID, c = i % HID;
        sWt2[r * LDH + c] = wt.Wt2[i];
        sWt3[r * LDH + c] = wt.Wt3[i];
        sW2[r * LDH + c] = wt.W2[i];
        sW3[r * LDH + c] = wt.W3[i];
    }
    for (int i = tid; i < 4 * HID + 1; i += blockDim.x) sb[i] = wt.bias[i];
    for (int i = lane; i < 4 * HID + 2; i += 32) sacc[warp][i] = 0.0f;
    __syncthreads();
    const float *b1 = sb, *b2 = sb + HID, *b3 = sb + 2 * HID, *w4 = sb + 3 * HID;
    const float b4 = sb[4 * HID];
    __nv_bfloat16 *sZ1 = sZ + (size_t)warp * ROWS_W * HID;
    __nv_bfloat16 *sZ2 = sZ + (size_t)(WARPS + warp) * ROWS_W * HID;

    const int64_t n_tiles = (src.R + ROWS_CTA - 1) / ROWS_CTA;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t r0 = tile * ROWS_CTA + warp * ROWS_W;
        const int64_t rA = r0 + g, rB = r0 + g + 8;
        float acc[16][4];
        uint32_t a[8][4];
        // ---- layer 1 (K = 16: 14 inputs and two zero columns)
        {
            float x[4][2];
            x[0][0] = in_val(src, rA, 2 * t);     x[0][1] = in_val(src, rA, 2 * t + 1);
            x[1][0] = in_val(src, rB, 2 * t);     x[1][1] = in_val(src, rB, 2 * t + 1);
            x[2][0] = in_val(src, rA, 2 * t + 8); x[2][1] = in_val(src, rA, 2 * t + 9);
            x[3][0] = in_val(src, rB, 2 * t + 8); x[3][1] = in_val(src, rB, 2 * t + 9);
            uint32_t a0[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) a0[q] = pack_bf16(x[q][0], x[q][1]);
            {
                const int64_t ld = tr.Rp;
                tr.H0[(size_t)(2 * t) * ld + rA] = __float2bfloat16_rn(x[0][0]);
                tr.H0[(size_t)(2 * t + 1) * ld + rA] = __float2bfloat16_rn(x[0][1]);
                tr.H0[(size_t)(2 * t) * ld + rB] = __float2bfloat16_rn(x[1][0]);
                tr.H0[(size_t)(2 * t + 1) * ld + rB] = __float2bfloat16_rn(x[1][1]);
                tr.H0[(size_t)(2 * t + 8) * ld + rA] = __float2bfloat16_rn(x[2][0]);
                tr.H0[(size_t)(2 * t + 9) * ld + rA] = __float2bfloat16_rn(x[2][1]);
                tr.H0[(size_t)(2 * t + 8) * ld + rB] = __float2bfloat16_rn(x[3][0]);
                tr.H0[(size_t)(2 * t + 9) * ld + rB] = __float2bfloat16_rn(x[3][1]);
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float c0 = b1[8 * j + 2 * t], c1 = b1[8 * j + 2 * t + 1];
                acc[j][0] = c0; acc[j][1] = c1; acc[j][2] = c0; acc[j][3] = c1;
                const __nv_bfloat16 *row = sWt1 + (8 * j + g) * LD1 + 2 * t;
                mma16816(acc[j], a0, *reinterpret_cast<const uint32_t *>(row),
                         *reinterpret_cast<const uint32_t *>(row + 8));
            }
        }
        // ---- layers 2 and 3; z_1, z_2 kept (BF16) for the backward pass
#pragma unroll 1
        for (int l = 1; l <= 2; ++l) {
            {
                __nv_bfloat16 *z = l == 1 ? sZ1 : sZ2;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    *reinterpret_cast<uint32_t *>(z + g * HID + 8 * j + 2 * t) = pack_bf16(acc[j][0], acc[j][1]);
                    *reinterpret_cast<uint32_t *>(z + (g + 8) * HID + 8 * j + 2 * t) = pack_bf16(acc[j][2], acc[j][3]);
                }
            }
#pragma unroll
            for (int j = 0; j < 16; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[j][q] = gelu(acc[j][q]);
            store_t(l == 1 ? tr.H1 : tr.H2, tr.Rp, r0, acc, g, t);
            to_frag(acc, a);
            const float *bb = l == 1 ? b2 : b3;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float c0 = bb[8 * j + 2 * t], c1 = bb[8 * j + 2 * t + 1];
                acc[j][0] = c0; acc[j][1] = c1; acc[j][2] = c0; acc[j][3] = c1;
            }
            gemm_128(acc, a, l == 1 ? sWt2 : sWt3, g, t);
        }
        // ---- output unit: o = GELU(z_3) . w4 + b4, t = softplus(o)
        float pA = 0.0f, pB = 0.0f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float u0 = w4[8 * j + 2 * t], u1 = w4[8 * j + 2 * t + 1];
            pA = fmaf(gelu(acc[j][0]), u0, fmaf(gelu(acc[j][1]), u1, pA));
            pB = fmaf(gelu(acc[j][2]), u0, fmaf(gelu(acc[j][3]), u1, pB));
        }
        pA += __shfl_xor_sync(0xffffffffu, pA, 1);
        pA += __shfl_xor_sync(0xffffffffu, pA, 2);
        pB += __shfl_xor_sync(0xffffffffu, pB, 1);
        pB += __shfl_xor_sync(0xffffffffu, pB, 2);
        const float oA = pA + b4, oB = pB + b4;
        const float yA = softplus(oA), yB = softplus(oB);
        // ---- loss and backward
        const bool vA = rA < src.R, vB = rB < src.R;
        const float eA = vA ? yA - src.target[rA] : 0.0f, eB = vB ? yB - src.target[rB] : 0.0f;
        const float doA = 2.0f * tr.inv_R * eA * sigmoid(oA), doB = 2.0f * tr.inv_R * eB * sigmoid(oB);
        {
            float l2 = (t == 0) ? eA * eA + eB * eB : 0.0f;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, o);
            float d4 = (t == 0) ? doA + doB : 0.0f;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) d4 += __shfl_xor_sync(0xffffffffu, d4, o);
            if (lane == 0) {
                sacc[warp][4 * HID] += d4;            // db4
                sacc[warp][4 * HID + 1] += l2;        // sum of squared errors
            }
        }
        // dw4 = sum_r h3 do, dz3 = do w4 GELU'(z3) (in place of z3)
        {
            float hw[16][4];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                hw[j][0] = gelu(acc[j][0]) * doA; hw[j][1] = gelu(acc[j][1]) * doA;
                hw[j][2] = gelu(acc[j][2]) * doB; hw[j][3] = gelu(acc[j][3]) * doB;
            }
            col_sums(hw, &sacc[warp][3 * HID], g, t);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float u0 = w4[8 * j + 2 * t], u1 = w4[8 * j + 2 * t + 1];
            acc[j][0] = doA * u0 * gelu_d(acc[j][0]);
            acc[j][1] = doA * u1 * gelu_d(acc[j][1]);
            acc[j][2] = doB * u0 * gelu_d(acc[j][2]);
            acc[j][3] = doB * u1 * gelu_d(acc[j][3]);
        }
#pragma unroll 1
        for (int l = 3; l >= 2; --l) {
            col_sums(acc, &sacc[warp][(l - 1) * HID], g, t);   // db_l
            store_t(l == 3 ? tr.dZ3 : tr.dZ2, tr.Rp, r0, acc, g, t);
            to_frag(acc, a);
#pragma unroll
            for (int j = 0; j < 16; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[j][q] = 0.0f;
            gemm_128(acc, a, l == 3 ? sW3 : sW2, g, t);   // dh_{l-1} = dz_l W_l^T
            const __nv_bfloat16 *z = l == 3 ? sZ2 : sZ1;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float2 zA = unpack_bf16(*reinterpret_cast<const uint32_t *>(z + g * HID + 8 * j + 2 * t));
                const float2 zB = unpack_bf16(*reinterpret_cast<const uint32_t *>(z + (g + 8) * HID + 8 * j + 2 * t));
                acc[j][0] *= gelu_d(zA.x);
                acc[j][1] *= gelu_d(zA.y);
                acc[j][2] *= gelu_d(zB.x);
                acc[j][3] *= gelu_d(zB.y);
            }
        }
        col_sums(acc, &sacc[warp][0], g, t);   // db1
        store_t(tr.dZ1, tr.Rp, r0, acc, g, t);
    }
    {
        __syncthreads();
        for (int i = tid; i < NPART; i += blockDim.x) {
            // partial layout: loss, db1, db2, db3, dw4, db4
            const int src_i = i == 0 ? 4 * HID + 1 : i - 1;
            float s = 0.0f;
            for (int w = 0; w < WARPS; ++w) s += sacc[w][src_i];
            tr.part[(size_t)blockIdx.x * NPART + i] = s;
        }
    }
}

// dW[k][n] partial over the rows [c * chunk, (c + 1) * chunk) of H^T [K][Rp] and dZ^T
// [128][Rp]: warp w computes rows k of its 16-row M tile (K = 128) or, for K = 16, the 16
// columns n of its slice.
__global__ void __launch_bounds__(WARPS * 32) k_mlp_dw(const __nv_bfloat16 *__restrict__ Ht,
                                                       const __nv_bfloat16 *__restrict__ dZt,
                                                       int32_t K, int64_t Rp, int64_t chunk,
                                                       float *__restrict__ part)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int m0 = K == HID ? 16 * warp : 0;
    const int n0 = K == HID ? 0 : 16 * warp;
    const int nt = K == HID ? 16 : 2;   // n-tiles of 8
    float acc[16][4];
#pragma unroll
    for (int j = 0; j < 16; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][q] = 0.0f;
    const int64_t beg = blockIdx.x * chunk, end = min(beg + chunk, Rp);
    for (int64_t r = beg; r < end; r += 16) {
        uint32_t a[4];
        const __nv_bfloat16 *ha = Ht + (size_t)(m0 + g) * Rp + r + 2 * t;
        const __nv_bfloat16 *hb = Ht + (size_t)(m0 + g + 8) * Rp + r + 2 * t;
        a[0] = *reinterpret_cast<const uint32_t *>(ha);
        a[1] = *reinterpret_cast<const uint32_t *>(hb);
        a[2] = *reinterpret_cast<const uint32_t *>(ha + 8);
        a[3] = *reinterpret_cast<const uint32_t *>(hb + 8);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j < nt) {
                const __nv_bfloat16 *bp = dZt + (size_t)(n0 + 8 * j + g) * Rp + r + 2 * t;
                mma16816(acc[j], a, *reinterpret_cast<const uint32_t *>(bp),
                         *reinterpret_cast<const uint32_t *>(bp + 8));
            }
        }
    }
    float *out = part + (size_t)blockIdx.x * K * HID;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j < nt) {
            const int c = n0 + 8 * j + 2 * t;
            out[(size_t)(m0 + g) * HID + c] = acc[j][0];
            out[(size_t)(m0 + g) * HID + c + 1] = acc[j][1];
            out[(size_t)(m0 + g + 8) * HID + c] = acc[j][2];
            out[(size_t)(m0 + g + 8) * HID + c + 1] = acc[j][3];
        }
    }
}

// grad[dst + i] = sum over c < n of part[c * stride + src + i] (fixed order), i < count;
// rows >= valid_rows of a [rows][128] block are skipped (W1's padding rows 14, 15).
__global__ void k_mlp_reduce(const float *__restrict__ part, int32_t n, int64_t stride,
                             int64_t src, int64_t count, float *__restrict__ grad, int64_t dst)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    float s = 0.0f;
    for (int c = 0; c < n; ++c) s += part[(size_t)c * stride + src + i];
    grad[dst + i] = s;
}

__global__ void k_mlp_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                           const float *__restrict__ grad, int32_t n, float lr, float b1,
                           float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------------------------ tcgen05 inference
// Operand images in shared memory, K-major with the 128-byte swizzle that the MMA descriptors
// name: a block holds 128 rows x 64 BF16 columns, row n at n * 128 bytes, its 16-byte chunk j
// (columns 8j .. 8j + 7) at (j xor (n mod 8)) * 16.  The weights' image is W1^T (one block,
// columns 14.. zero), W2^T and W3^T (two blocks each), built by k_mlp_pack in global memory and
// copied whole by the TMA unit; a tile's activations H (128 rows x 128 columns) are two blocks.
constexpr uint32_t BLK = HID * 128;                           // bytes of one block: 16 KB
constexpr uint32_t IMG_W1 = 0, IMG_W2 = BLK, IMG_W3 = 3 * BLK, IMG_BYTES = 5 * BLK;
constexpr int TC_GROUPS = 3;                                  // 128-row tiles in flight per CTA
constexpr int TC_THREADS = TC_GROUPS * 128;                   // one thread per row of a tile
constexpr size_t TC_SMEM = IMG_BYTES + (size_t)TC_GROUPS * 2 * BLK + 1024;   // + alignment
constexpr uint32_t TC_TMEM_COLS = TC_GROUPS * HID <= 256 ? 256 : 512;   // a power of two holding
                                                                          // one accumulator per group
static_assert(TC_GROUPS * HID <= 512, "TMEM columns");
constexpr long long kMlpWaitNs = 1000000000LL;                // 1 s per wait, then an error

// Byte offset of element (row, col) in a stack of blocks (col / 64 selects the block).
__host__ __device__ __forceinline__ uint32_t swz(uint32_t row, uint32_t col)
{
    return (col >> 6) * BLK + row * 128 + ((((col & 63) >> 3) ^ (row & 7)) << 4) + (col & 7) * 2;
}

__device__ __forceinline__ void img_put(uint8_t *img, uint32_t base, int n, int k, float v)
{
    *reinterpret_cast<__nv_bfloat16 *>(img + base + swz((uint32_t)n, (uint32_t)k)) = __float2bfloat16_rn(v);
}

__device__ __forceinline__ void tmem_ld_wait16(uint32_t (&a)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]),
                   "+r"(a[6]), "+r"(a[7]), "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]),
                   "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15])
                 :
                 : "memory");
}

// The 14 inputs of row r (two zero columns after them; zeros past the row count) into the
// tile's first block, BF16.
__device__ __forceinline__ void put_inputs(const RowSrc &s, int64_t r, uint8_t *sH, uint32_t row)
{
    float x[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) x[c] = 0.0f;
    if (r < s.R) {
        int64_t fr, wr;
        if (s.pairs) {
            fr = s.pairs[2 * r];
            wr = s.pairs[2 * r + 1];
        } else {
            fr = r % s.n_dwell;
            wr = r / s.n_dwell;
        }
#pragma unroll
        for (int c = 0; c < NFEAT; ++c) x[c] = s.feat[fr * NFEAT + c];
#pragma unroll
        for (int c = 0; c < NW; ++c) x[NFEAT + c] = log10f(fmaxf(s.w[wr * NW + c], 1e-3f));
    }
    uint4 lo, hi;
    lo.x = pack_bf16(x[0], x[1]);   lo.y = pack_bf16(x[2], x[3]);
    lo.z = pack_bf16(x[4], x[5]);   lo.w = pack_bf16(x[6], x[7]);
    hi.x = pack_bf16(x[8], x[9]);   hi.y = pack_bf16(x[10], x[11]);
    hi.z = pack_bf16(x[12], x[13]); hi.w = pack_bf16(x[14], x[15]);
    *reinterpret_cast<uint4 *>(sH + swz(row, 0)) = lo;
    *reinterpret_cast<uint4 *>(sH + swz(row, 8)) = hi;
}

// Hidden-layer epilogue of one row: h = GELU(z + b) from the accumulator's 128 columns
// (TMEM lane = row), BF16 into the tile's blocks as the next layer's A operand.  32 columns
// per pass, the passes not unrolled: the GELUs of the whole row unrolled would not fit the
// instruction cache.
__device__ __forceinline__ void epi_hidden(uint32_t taddr, const float *b, uint8_t *sH, uint32_t row)
{
#pragma unroll 1
    for (int c0 = 0; c0 < HID; c0 += 32) {
        uint32_t v[2][16];
        gmco::tmem_ld16(taddr + (uint32_t)c0, v[0]);
        gmco::tmem_ld16(taddr + (uint32_t)c0 + 16, v[1]);
        tmem_ld_wait16(v[0]);
        tmem_ld_wait16(v[1]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t h[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = 8 * q + 2 * e;   // column c0 + c of the pass
                h[e] = pack_bf16(gelu(__uint_as_float(v[c >> 4][c & 15]) + b[c0 + c]),
                                 gelu(__uint_as_float(v[c >> 4][(c & 15) + 1]) + b[c0 + c + 1]));
            }
            *reinterpret_cast<uint4 *>(sH + swz(row, (uint32_t)(c0 + 8 * q))) = make_uint4(h[0], h[1], h[2], h[3]);
        }
    }
}

// Output unit of one row: o = sum_c GELU(z_3c + b_3c) w_4c (FP32, in column order) + b_4.
__device__ __forceinline__ float epi_out(uint32_t taddr, const float *b3, const float *w4, float b4)
{
    float o = 0.0f;
#pragma unroll 1
    for (int c0 = 0; c0 < HID; c0 += 32) {
        uint32_t v[2][16];
        gmco::tmem_ld16(taddr + (uint32_t)c0, v[0]);
        gmco::tmem_ld16(taddr + (uint32_t)c0 + 16, v[1]);
        tmem_ld_wait16(v[0]);
        tmem_ld_wait16(v[1]);
#pragma unroll
        for (int c = 0; c < 32; ++c)
            o = fmaf(gelu(__uint_as_float(v[c >> 4][c & 15]) + b3[c0 + c]), w4[c0 + c], o);
    }
    return o + b4;
}

// Forward pass of the network for inference on the fifth-generation tensor cores.  Persistent
// CTAs of TC_GROUPS groups of four warps; a group owns one 128-row tile at a time (thread =
// row = TMEM lane), 128 accumulator columns of TMEM and two activation blocks.  Per tile: the
// threads write the inputs, one elected thread issues the layer's tcgen05.mma (M = N = 128,
// K = 16 for layer 1, 128 for layers 2 and 3) and commits it to the group's mbarrier, the
// threads read the accumulator with tcgen05.ld, add the bias, apply GELU and write BF16
// activations for the next layer; the output unit and softplus finish in registers.  The
// groups interleave, so one group's MMAs run under the others' epilogues.  Every wait is
// bounded: a wait that runs out sets *err, the group stops at its next barrier, and the CTA
// waits (bounded) for its MMAs and copies in flight before freeing TMEM.
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_mlp_infer_tc(const uint8_t *__restrict__ img, const float *__restrict__ bias, RowSrc src,
                   float t_floor, float *__restrict__ t_out, int32_t *__restrict__ err)
{
    using namespace gmco;
    extern __shared__ uint8_t dyn[];
    __shared__ float sb[4 * HID + 1];
    __shared__ __align__(8) uint64_t w_bar, mma_bar[TC_GROUPS], drain_bar[TC_GROUPS];
    __shared__ uint32_t tmem_holder;
    uint8_t *base = reinterpret_cast<uint8_t *>(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = warp >> 2;
    const uint32_t row = (uint32_t)(32 * (warp & 3) + lane);
    const bool issuer = (warp & 3) == 0;   // the group's first warp issues its MMAs
    const uint32_t s_img = smem_u32(base);
    uint8_t *sH = base + IMG_BYTES + (size_t)grp * 2 * BLK;
    const uint32_t s_h = smem_u32(sH);

    if (tid == 0) {
        mbar_init(smem_u32(&w_bar), 1);
        for (int g = 0; g < TC_GROUPS; ++g) {
            mbar_init(smem_u32(&mma_bar[g]), 1);
            mbar_init(smem_u32(&drain_bar[g]), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_holder), TC_TMEM_COLS);
    for (int i = tid; i < 4 * HID + 1; i += TC_THREADS) sb[i] = bias[i];
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_holder;
    if (tid == 0) {
        mbar_expect_tx(smem_u32(&w_bar), IMG_BYTES);
        for (uint32_t c = 0; c < IMG_BYTES / BLK; ++c) bulk_load(s_img + c * BLK, img + c * BLK, BLK, smem_u32(&w_bar));
    }
    const bool w_ok = mbar_wait(smem_u32(&w_bar), 0u, err, 1, kMlpWaitNs);
    const bool w_fail = __syncthreads_or(!w_ok);
    if (w_fail && tid == 0) mbar_wait(smem_u32(&w_bar), 0u, nullptr, 0, kMlpWaitNs);   // copies in flight

    const uint32_t d_col = tmem + (uint32_t)(grp * HID);           // accumulator (lane 0)
    const uint32_t t_row = d_col + ((uint32_t)(32 * (warp & 3)) << 16);   // this warp's lanes
    const uint32_t idesc = idesc_bf16(HID);
    const uint32_t bar = smem_u32(&mma_bar[grp]);
    const float *b1 = sb, *b2 = sb + HID, *b3 = sb + 2 * HID, *w4 = sb + 3 * HID;
    const float b4 = sb[4 * HID];
    const int64_t n_tiles = (src.R + 127) / 128;
    uint32_t parity = 0;
    bool pending = false;   // this thread's last MMA wait gave up
    bool failed = w_fail;   // uniform over the group
    for (int64_t tile = (int64_t)blockIdx.x * TC_GROUPS + grp; !failed && tile < n_tiles;
         tile += (int64_t)gridDim.x * TC_GROUPS) {
        const int64_t r = tile * 128 + row;
        put_inputs(src, r, sH, row);
        float o = 0.0f;
#pragma unroll 1
        for (int l = 0; l < 3; ++l) {
            // the threads' operand writes and TMEM reads are done before the MMAs start
            fence_proxy_async_smem();
            fence_before();
            if (bar_any(1 + grp, 128, pending)) {
                failed = true;
                break;
            }
            if (issuer) {
                fence_after();
                if (l == 0) {
                    mma_bf16_elect(d_col, DESC_FIXED | desc_lo(s_h), DESC_FIXED | desc_lo(s_img + IMG_W1), idesc, 0u);
                } else {
                    const uint32_t wb = s_img + (l == 1 ? IMG_W2 : IMG_W3);
#pragma unroll
                    for (int k = 0; k < HID / 16; ++k) {
                        const uint32_t off = (uint32_t)(k >> 2) * BLK + (uint32_t)(k & 3) * 32;
                        mma_bf16_elect(d_col, DESC_FIXED | desc_lo(s_h + off), DESC_FIXED | desc_lo(wb + off),
                                       idesc, k > 0 ? 1u : 0u);
                    }
                }
                mma_commit_elect(bar);
            }
            pending = !mbar_wait(bar, parity, err, 2, kMlpWaitNs);
            parity ^= 1u;
            fence_after();
            if (l < 2) epi_hidden(t_row, l == 0 ? b1 : b2, sH, row);
            else o = epi_out(t_row, b3, w4, b4);
        }
        if (!failed && r < src.R) t_out[r] = fmaxf(softplus(o), t_floor);
    }
    fence_before();
    if (!failed) failed = bar_any(1 + grp, 128, pending);
    if (failed && !w_fail && issuer) {
        // MMAs issued before a wait gave up may still be running: their commit completes once
        // they have all finished
        mma_commit_elect(smem_u32(&drain_bar[grp]));
        mbar_wait(smem_u32(&drain_bar[grp]), 0u, nullptr, 0, kMlpWaitNs);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        tmem_dealloc(tmem, TC_TMEM_COLS);
    }
}

// BF16 copies of the FP32 master parameters in the kernels' layouts.
__global__ void k_mlp_pack(const float *__restrict__ p, DevWeights w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < HID * HID) {
        const int k = i / HID, n = i % HID;   // W[k][n]
        w.W2[i] = __float2bfloat16_rn(p[OFF_W2 + i]);
        w.W3[i] = __float2bfloat16_rn(p[OFF_W3 + i]);
        w.Wt2[n * HID + k] = __float2bfloat16_rn(p[OFF_W2 + i]);
        w.Wt3[n * HID + k] = __float2bfloat16_rn(p[OFF_W3 + i]);
    }
    if (i < HID * KIN) {
        const int n = i / KIN, k = i % KIN;   // Wt1[n][k]
        w.Wt1[i] = __float2bfloat16_rn(k < NIN ? p[OFF_W1 + k * HID + n] : 0.0f);
    }
    if (i < HID * 64) {
        const int n = i / 64, k = i % 64;     // one 64-column block of W1^T, columns 14.. zero
        img_put(w.img, IMG_W1, n, k, k < NIN ? p[OFF_W1 + k * HID + n] : 0.0f);
    }
    if (i < HID * HID) {
        const int k = i / HID, n = i % HID;
        img_put(w.img, IMG_W2, n, k, p[OFF_W2 + i]);
        img_put(w.img, IMG_W3, n, k, p[OFF_W3 + i]);
    }
    if (i < 4 * HID + 1) {
        // bias[] = b1, b2, b3, w4 (128 each), then b4
        const int blk = i / HID, o = i % HID;
        const int srcs[4] = {OFF_B1, OFF_B2, OFF_B3, OFF_W4};
        w.bias[i] = i == 4 * HID ? p[OFF_B4] : p[srcs[blk] + o];
    }
}

size_t train_smem()
{
    return (size_t)HID * LD1 * 2 + 4 * (size_t)HID * LDH * 2 + 2 * (size_t)WARPS * ROWS_W * HID * 2;
}

thread_local std::string g_mlp_err;

}  // namespace

struct gmco_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<void *> allocs;
    float *p = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;   // FP32, NPARAM each
    DevWeights w{};
    int32_t *err = nullptr;   // wait status of the inference kernel (0 = none ran out)
    int64_t step = 0;
    // training workspace
    int64_t cap_rows = 0;
    TrainOut tr{};
    float *dwpart = nullptr;
    int32_t n_dw_cta = 0;
    // staging of host inputs
    std::vector<void *> ws;
    float *h_pinned = nullptr;
    int64_t launches = 0;
};

namespace {

#define MCK(call)                                                                   \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            g_mlp_err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
            return e_ == cudaErrorMemoryAllocation ? GMCO_ENOMEM : GMCO_ECUDA;      \
        }                                                                           \
    } while (0)

template <class T>
cudaError_t dalloc(gmco_mlp *q, T **p, size_t n, bool ws = false)
{
    void *r = nullptr;
    cudaError_t e = cudaMalloc(&r, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    (ws ? q->ws : q->allocs).push_back(r);
    *p = static_cast<T *>(r);
    return cudaSuccess;
}

void free_ws(gmco_mlp *q)
{
    for (void *p : q->ws) cudaFree(p);
    q->ws.clear();
    q->cap_rows = 0;
}

gmco_status pack(gmco_mlp *q)
{
    k_mlp_pack<<<(HID * HID + 255) / 256, 256, 0, q->stream>>>(q->p, q->w);
    MCK(cudaGetLastError());
    q->launches++;
    return GMCO_OK;
}

// Device copies of (possibly host) inputs, in a per-call arena.
struct Staged {
    std::vector<void *> ptrs;
    ~Staged()
    {
        for (void *p : ptrs) cudaFree(p);
    }
};

template <class T>
gmco_status stage(gmco_mlp *q, Staged &s, const T *src, size_t n, const T **out)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, src) == cudaSuccess &&
        (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
        *out = src;
        return GMCO_OK;
    }
    cudaGetLastError();
    void *d = nullptr;
    MCK(cudaMalloc(&d, std::max<size_t>(n, 1) * sizeof(T)));
    s.ptrs.push_back(d);
    MCK(cudaMemcpyAsync(d, src, n * sizeof(T), cudaMemcpyHostToDevice, q->stream));
    *out = static_cast<const T *>(d);
    return GMCO_OK;
}

gmco_status begin(gmco_mlp *q, void *user_stream)
{
    MCK(cudaSetDevice(q->device));
    MCK(cudaEventRecord(q->ev_in, (cudaStream_t)user_stream));
    MCK(cudaStreamWaitEvent(q->stream, q->ev_in, 0));
    return GMCO_OK;
}

gmco_status finish(gmco_mlp *q, void *user_stream)
{
    MCK(cudaEventRecord(q->ev_out, q->stream));
    MCK(cudaStreamWaitEvent((cudaStream_t)user_stream, q->ev_out, 0));
    MCK(cudaStreamSynchronize(q->stream));
    return GMCO_OK;
}

int n_ctas(int64_t R) { return (int)std::min<int64_t>(MAX_CTAS, std::max<int64_t>(1, (R + ROWS_CTA - 1) / ROWS_CTA)); }

// Loss and gradient (into q->grad) of the batch at the current BF16 weights.
gmco_status gradient(gmco_mlp *q, const RowSrc &src, float *loss_out)
{
    const int64_t R = src.R;
    const int64_t Rp = (R + ROWS_CTA - 1) / ROWS_CTA * ROWS_CTA;
    if (Rp > q->cap_rows) {
        MCK(cudaStreamSynchronize(q->stream));
        free_ws(q);
        TrainOut &t = q->tr;
        MCK(dalloc(q, &t.H0, (size_t)KIN * Rp, true));
        MCK(dalloc(q, &t.H1, (size_t)HID * Rp, true));
        MCK(dalloc(q, &t.H2, (size_t)HID * Rp, true));
        MCK(dalloc(q, &t.dZ1, (size_t)HID * Rp, true));
        MCK(dalloc(q, &t.dZ2, (size_t)HID * Rp, true));
        MCK(dalloc(q, &t.dZ3, (size_t)HID * Rp, true));
        MCK(dalloc(q, &t.part, (size_t)MAX_CTAS * NPART, true));
        MCK(dalloc(q, &q->dwpart, (size_t)MAX_CTAS * HID * HID, true));
        q->cap_rows = Rp;
    }
    TrainOut tr = q->tr;
    tr.Rp = Rp;
    tr.inv_R = 1.0f / (float)R;
    // rows R..Rp of the feature-major arrays are written by the kernel (tiles cover Rp)
    const int ctas = n_ctas(R);
    const size_t smem = train_smem();
    MCK(cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RowSrc s2 = src;
    k_mlp_train<<<ctas, WARPS * 32, smem, q->stream>>>(q->w, s2, tr);
    MCK(cudaGetLastError());
    q->launches++;
    // bias and output-unit gradients, loss
    const int rb = 256;
    k_mlp_reduce<<<(HID + rb - 1) / rb, rb, 0, q->stream>>>(tr.part, ctas, NPART, 1, HID, q->grad, OFF_B1);
    k_mlp_reduce<<<(HID + rb - 1) / rb, rb, 0, q->stream>>>(tr.part, ctas, NPART, 1 + HID, HID, q->grad, OFF_B2);
    k_mlp_reduce<<<(HID + rb - 1) / rb, rb, 0, q->stream>>>(tr.part, ctas, NPART, 1 + 2 * HID, HID, q->grad, OFF_B3);
    k_mlp_reduce<<<(HID + 1 + rb - 1) / rb, rb, 0, q->stream>>>(tr.part, ctas, NPART, 1 + 3 * HID, HID + 1, q->grad, OFF_W4);
    MCK(cudaGetLastError());
    q->launches += 4;
    // weight gradients, split over row ranges
    const int64_t chunk = std::max<int64_t>(16, (Rp / MAX_CTAS + 15) / 16 * 16);
    const int nd = (int)((Rp + chunk - 1) / chunk);
    struct L { const __nv_bfloat16 *H, *dZ; int K; int off; };
    const L layers[3] = {{tr.H0, tr.dZ1, KIN, OFF_W1}, {tr.H1, tr.dZ2, HID, OFF_W2}, {tr.H2, tr.dZ3, HID, OFF_W3}};
    for (const L &l : layers) {
        k_mlp_dw<<<nd, WARPS * 32, 0, q->stream>>>(l.H, l.dZ, l.K, Rp, chunk, q->dwpart);
        const int64_t cnt = (int64_t)(l.K == KIN ? NIN : HID) * HID;   // W1: rows 0..13 only
        k_mlp_reduce<<<(unsigned)((cnt + rb - 1) / rb), rb, 0, q->stream>>>(q->dwpart, nd, (int64_t)l.K * HID,
                                                                           0, cnt, q->grad, l.off);
        MCK(cudaGetLastError());
        q->launches += 2;
    }
    if (loss_out) {
        k_mlp_reduce<<<1, 32, 0, q->stream>>>(tr.part, ctas, NPART, 0, 1, q->grad + NPARAM, 0);
        MCK(cudaGetLastError());
        q->launches++;
        MCK(cudaMemcpyAsync(q->h_pinned, q->grad + NPARAM, sizeof(float), cudaMemcpyDeviceToHost, q->stream));
        MCK(cudaStreamSynchronize(q->stream));
        *loss_out = q->h_pinned[0] / (float)R;
    }
    return GMCO_OK;
}

gmco_status batch_args(gmco_mlp *q, Staged &st, const float *feat, int64_t n_feat,
                       const float *w, int64_t n_w, const int32_t *pairs, const float *target,
                       int64_t R, RowSrc *src)
{
    if (!feat || !w || !pairs || !target || n_feat < 1 || n_w < 1 || R < 1 || R > (1LL << 26)) {
        g_mlp_err = "bad training batch";
        return GMCO_EINVAL;
    }
    RowSrc s{};
    gmco_status r;
    if ((r = stage(q, st, feat, (size_t)n_feat * NFEAT, &s.feat)) != GMCO_OK) return r;
    if ((r = stage(q, st, w, (size_t)n_w * NW, &s.w)) != GMCO_OK) return r;
    if ((r = stage(q, st, pairs, (size_t)R * 2, &s.pairs)) != GMCO_OK) return r;
    if ((r = stage(q, st, target, (size_t)R, &s.target)) != GMCO_OK) return r;
    // index check on the host copy of the pairs
    std::vector<int32_t> hp((size_t)R * 2);
    MCK(cudaMemcpyAsync(hp.data(), s.pairs, hp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, q->stream));
    MCK(cudaStreamSynchronize(q->stream));
    for (int64_t i = 0; i < R; ++i)
        if (hp[2 * i] < 0 || hp[2 * i] >= n_feat || hp[2 * i + 1] < 0 || hp[2 * i + 1] >= n_w) {
            g_mlp_err = "pair index out of range";
            return GMCO_EINVAL;
        }
    s.n_dwell = 0;
    s.R = R;
    *src = s;
    return GMCO_OK;
}

}  // namespace

extern "C" {

const char *gmco_mlp_last_error(void) { return g_mlp_err.c_str(); }

void gmco_mlp_destroy(gmco_mlp *q)
{
    if (!q) return;
    cudaSetDevice(q->device);
    if (q->stream) cudaStreamSynchronize(q->stream);
    free_ws(q);
    for (void *p : q->allocs) cudaFree(p);
    if (q->h_pinned) cudaFreeHost(q->h_pinned);
    if (q->ev_in) cudaEventDestroy(q->ev_in);
    if (q->ev_out) cudaEventDestroy(q->ev_out);
    if (q->stream) cudaStreamDestroy(q->stream);
    delete q;
}

gmco_status gmco_mlp_create(const float *params, gmco_mlp **out)
{
    if (!out) return GMCO_EINVAL;
    *out = nullptr;
    if (!params) {
        g_mlp_err = "gmco_mlp_create: null parameters";
        return GMCO_EINVAL;
    }
    int nd = 0;
    if (cudaGetDeviceCount(&nd) != cudaSuccess || nd < 1) {
        cudaGetLastError();
        g_mlp_err = "gmco_mlp_create: no CUDA device";
        return GMCO_ECUDA;
    }
    std::vector<float> hp(NPARAM);
    if (cudaMemcpy(hp.data(), params, NPARAM * sizeof(float), cudaMemcpyDefault) != cudaSuccess) {
        cudaGetLastError();
        g_mlp_err = "gmco_mlp_create: cannot read parameters";
        return GMCO_EINVAL;
    }
    for (float x : hp)
        if (!std::isfinite(x)) {
            g_mlp_err = "gmco_mlp_create: non-finite parameter";
            return GMCO_EINVAL;
        }
    gmco_mlp *q = new gmco_mlp();
    cudaGetDevice(&q->device);
    auto fail = [&](gmco_status s) {
        gmco_mlp_destroy(q);
        return s;
    };
    if (cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&q->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&q->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&q->h_pinned, 64) != cudaSuccess)
        return fail(GMCO_ECUDA);
    if (dalloc(q, &q->p, NPARAM) != cudaSuccess || dalloc(q, &q->m, NPARAM) != cudaSuccess ||
        dalloc(q, &q->v, NPARAM) != cudaSuccess || dalloc(q, &q->grad, NPARAM + 1) != cudaSuccess ||
        dalloc(q, &q->w.Wt1, HID * KIN) != cudaSuccess || dalloc(q, &q->w.Wt2, HID * HID) != cudaSuccess ||
        dalloc(q, &q->w.Wt3, HID * HID) != cudaSuccess || dalloc(q, &q->w.W2, HID * HID) != cudaSuccess ||
        dalloc(q, &q->w.W3, HID * HID) != cudaSuccess || dalloc(q, &q->w.bias, 4 * HID + 1) != cudaSuccess ||
        dalloc(q, &q->w.img, IMG_BYTES) != cudaSuccess || dalloc(q, &q->err, 1) != cudaSuccess)
        return fail(GMCO_ENOMEM);
    if (cudaMemcpy(q->p, hp.data(), NPARAM * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(q->m, 0, NPARAM * sizeof(float)) != cudaSuccess ||
        cudaMemset(q->v, 0, NPARAM * sizeof(float)) != cudaSuccess ||
        cudaMemset(q->grad, 0, (NPARAM + 1) * sizeof(float)) != cudaSuccess ||
        cudaMemset(q->err, 0, sizeof(int32_t)) != cudaSuccess)
        return fail(GMCO_ECUDA);
    if (pack(q) != GMCO_OK || cudaStreamSynchronize(q->stream) != cudaSuccess) return fail(GMCO_ECUDA);
    *out = q;
    return GMCO_OK;
}

gmco_status gmco_mlp_get_params(gmco_mlp *q, float *params)
{
    if (!q || !params) return GMCO_EINVAL;
    MCK(cudaSetDevice(q->device));
    MCK(cudaStreamSynchronize(q->stream));
    MCK(cudaMemcpy(params, q->p, NPARAM * sizeof(float), cudaMemcpyDefault));
    return GMCO_OK;
}

// Checkpoint file: the line "GMCO-MLP", one line of JSON describing the contents, then three
// arrays of GMCO_MLP_NPARAM little-endian FP32 values: the master parameters, Adam's first and
// second moments.  The header carries the Adam step count, the format version and the layout.
static const char kMlpMagic[] = "GMCO-MLP\n";

gmco_status gmco_mlp_save(gmco_mlp *q, const char *path)
{
    if (!q || !path) {
        g_mlp_err = "gmco_mlp_save: bad arguments";
        return GMCO_EINVAL;
    }
    std::vector<float> buf((size_t)3 * NPARAM);
    MCK(cudaSetDevice(q->device));
    MCK(cudaStreamSynchronize(q->stream));
    MCK(cudaMemcpy(buf.data(), q->p, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    MCK(cudaMemcpy(buf.data() + NPARAM, q->m, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    MCK(cudaMemcpy(buf.data() + 2 * (size_t)NPARAM, q->v, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    FILE *f = fopen(path, "wb");
    if (!f) {
        g_mlp_err = std::string("gmco_mlp_save: cannot open ") + path;
        return GMCO_EINVAL;
    }
    char hdr[512];
    snprintf(hdr, sizeof hdr,
             "{\"format\": \"gmco-mlp\", \"version\": 1, \"nparam\": %d, \"step\": %lld, "
             "\"arrays\": [\"params\", \"adam_m\", \"adam_v\"], \"dtype\": \"float32-le\", "
             "\"adam\": {\"beta1\": 0.9, \"beta2\": 0.999, \"eps\": 1e-08}, "
             "\"layout\": [[\"W1\", 14, 128], [\"b1\", 128], [\"W2\", 128, 128], [\"b2\", 128], "
             "[\"W3\", 128, 128], [\"b3\", 128], [\"w4\", 128], [\"b4\", 1]]}\n",
             (int)NPARAM, (long long)q->step);
    const bool ok = fputs(kMlpMagic, f) >= 0 && fputs(hdr, f) >= 0 &&
                    fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    if (fclose(f) != 0 || !ok) {
        g_mlp_err = std::string("gmco_mlp_save: write failed for ") + path;
        return GMCO_EINVAL;
    }
    return GMCO_OK;
}

gmco_status gmco_mlp_load(const char *path, gmco_mlp **out)
{
    if (!out) return GMCO_EINVAL;
    *out = nullptr;
    if (!path) {
        g_mlp_err = "gmco_mlp_load: bad arguments";
        return GMCO_EINVAL;
    }
    FILE *f = fopen(path, "rb");
    if (!f) {
        g_mlp_err = std::string("gmco_mlp_load: cannot open ") + path;
        return GMCO_EINVAL;
    }
    char magic[16] = {0}, hdr[1024] = {0};
    std::vector<float> buf((size_t)3 * NPARAM);
    bool ok = fgets(magic, sizeof magic, f) && strcmp(magic, kMlpMagic) == 0 && fgets(hdr, sizeof hdr, f);
    long long step = -1, nparam = -1, version = -1;
    if (ok) {
        const char *a = strstr(hdr, "\"nparam\":"), *b = strstr(hdr, "\"step\":"),
                   *c = strstr(hdr, "\"version\":");
        ok = a && b && c && strstr(hdr, "\"float32-le\"");
        if (ok) {
            nparam = strtoll(a + 9, nullptr, 10);
            step = strtoll(b + 7, nullptr, 10);
            version = strtoll(c + 10, nullptr, 10);
        }
        ok = ok && version == 1 && nparam == NPARAM && step >= 0;
    }
    ok = ok && fread(buf.data(), sizeof(float), buf.size(), f) == buf.size() && fgetc(f) == EOF;
    fclose(f);
    if (!ok) {
        g_mlp_err = std::string("gmco_mlp_load: not a version-1 checkpoint of this network: ") + path;
        return GMCO_EINVAL;
    }
    for (size_t i = 0; i < buf.size(); ++i)
        if (!std::isfinite(buf[i]) || (i >= 2 * (size_t)NPARAM && buf[i] < 0.0f)) {
            g_mlp_err = "gmco_mlp_load: non-finite value or negative second moment";
            return GMCO_EINVAL;
        }
    gmco_mlp *q = nullptr;
    gmco_status r = gmco_mlp_create(buf.data(), &q);
    if (r != GMCO_OK) return r;
    if (cudaMemcpy(q->m, buf.data() + NPARAM, NPARAM * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(q->v, buf.data() + 2 * (size_t)NPARAM, NPARAM * sizeof(float), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        g_mlp_err = "gmco_mlp_load: cannot copy the optimiser state";
        gmco_mlp_destroy(q);
        return GMCO_ECUDA;
    }
    q->step = step;
    *out = q;
    return GMCO_OK;
}

int64_t gmco_mlp_last_launch_count(const gmco_mlp *q) { return q ? q->launches : -1; }

gmco_status gmco_mlp_predict(gmco_mlp *q, const float *features, int64_t n_dwell,
                             const float *penalty_weights, int64_t P, float t_floor,
                             float *t_out, void *cuda_stream)
{
    if (!q || !features || !penalty_weights || !t_out || n_dwell < 1 || P < 1 ||
        n_dwell * P > (1LL << 31) || !(t_floor >= 0.0f) || !std::isfinite(t_floor)) {
        g_mlp_err = "gmco_mlp_predict: bad arguments";
        return GMCO_EINVAL;
    }
    q->launches = 0;
    gmco_status r;
    if ((r = begin(q, cuda_stream)) != GMCO_OK) return r;
    Staged st;
    RowSrc s{};
    if ((r = stage(q, st, features, (size_t)n_dwell * NFEAT, &s.feat)) != GMCO_OK) return r;
    if ((r = stage(q, st, penalty_weights, (size_t)P * NW, &s.w)) != GMCO_OK) return r;
    s.pairs = nullptr;
    s.n_dwell = n_dwell;
    s.R = n_dwell * P;
    float *dst = t_out;
    cudaPointerAttributes a{};
    const bool dev_out = cudaPointerGetAttributes(&a, t_out) == cudaSuccess &&
                         (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (!dev_out) {
        void *d = nullptr;
        MCK(cudaMalloc(&d, (size_t)s.R * sizeof(float)));
        st.ptrs.push_back(d);
        dst = static_cast<float *>(d);
    }
    int n_sm = 0;
    MCK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, q->device));
    const int64_t n_tiles = (s.R + 127) / 128;
    const int ctas = (int)std::min<int64_t>(n_sm, (n_tiles + TC_GROUPS - 1) / TC_GROUPS);
    MCK(cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    k_mlp_infer_tc<<<ctas, TC_THREADS, TC_SMEM, q->stream>>>(q->w.img, q->w.bias, s, t_floor, dst, q->err);
    MCK(cudaGetLastError());
    q->launches++;
    if (!dev_out)
        MCK(cudaMemcpyAsync(t_out, dst, (size_t)s.R * sizeof(float), cudaMemcpyDeviceToHost, q->stream));
    MCK(cudaMemcpyAsync(q->h_pinned + 1, q->err, sizeof(int32_t), cudaMemcpyDeviceToHost, q->stream));
    if ((r = finish(q, cuda_stream)) != GMCO_OK) return r;
    int32_t code = 0;
    memcpy(&code, q->h_pinned + 1, sizeof code);
    if (code != 0) {
        // a bounded wait of the kernel ran out: the predictions are not valid
        cudaMemsetAsync(q->err, 0, sizeof(int32_t), q->stream);
        cudaStreamSynchronize(q->stream);
        g_mlp_err = "gmco_mlp_predict: a tensor-core wait of the inference kernel ran out (code " +
                    std::to_string(code) + ")";
        return GMCO_ECUDA;
    }
    return GMCO_OK;
}

gmco_status gmco_mlp_gradient(gmco_mlp *q, const float *features, int64_t n_feat,
                              const float *penalty_weights, int64_t n_w, const int32_t *pairs,
                              const float *target, int64_t R, float *loss, float *grad,
                              void *cuda_stream)
{
    if (!q || !grad) {
        g_mlp_err = "gmco_mlp_gradient: bad arguments";
        return GMCO_EINVAL;
    }
    q->launches = 0;
    gmco_status r;
    if ((r = begin(q, cuda_stream)) != GMCO_OK) return r;
    Staged st;
    RowSrc s{};
    if ((r = batch_args(q, st, features, n_feat, penalty_weights, n_w, pairs, target, R, &s)) != GMCO_OK)
        return r;
    float l = 0.0f;
    if ((r = gradient(q, s, &l)) != GMCO_OK) return r;
    if (loss) *loss = l;
    MCK(cudaMemcpyAsync(grad, q->grad, NPARAM * sizeof(float), cudaMemcpyDefault, q->stream));
    return finish(q, cuda_stream);
}

gmco_status gmco_mlp_train_step(gmco_mlp *q, const float *features, int64_t n_feat,
                                const float *penalty_weights, int64_t n_w, const int32_t *pairs,
                                const float *target, int64_t R, float lr, float *loss,
                                void *cuda_stream)
{
    if (!q || !(lr > 0.0f) || !std::isfinite(lr)) {
        g_mlp_err = "gmco_mlp_train_step: bad arguments";
        return GMCO_EINVAL;
    }
    q->launches = 0;
    gmco_status r;
    if ((r = begin(q, cuda_stream)) != GMCO_OK) return r;
    Staged st;
    RowSrc s{};
    if ((r = batch_args(q, st, features, n_feat, penalty_weights, n_w, pairs, target, R, &s)) != GMCO_OK)
        return r;
    float l = 0.0f;
    if ((r = gradient(q, s, loss ? &l : nullptr)) != GMCO_OK) return r;
    q->step++;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - (float)pow((double)b1, (double)q->step);
    const float c2 = 1.0f - (float)pow((double)b2, (double)q->step);
    k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, q->stream>>>(q->p, q->m, q->v, q->grad, NPARAM, lr,
                                                          b1, b2, eps, c1, c2);
    MCK(cudaGetLastError());
    q->launches++;
    if ((r = pack(q)) != GMCO_OK) return r;
    if (loss) *loss = l;
    return finish(q, cuda_stream);
}

}  // extern "C"
