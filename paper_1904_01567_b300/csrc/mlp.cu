// Learned warm start: a per-dwell-position multilayer perceptron that maps 10 geometric
// features of a dwell position and the 4 penalty weights of a plan to a dwell time,
//     x0 = [f_1..f_10, log10 max(w_1, 1e-3) .. log10 max(w_4, 1e-3)]      (14 inputs)
//     h_l = GELU(h_{l-1} W_l + b_l), l = 1, 2, 3 (width 128, GELU(z) = z Phi(z) with erf)
//     t = softplus(h_3 . w_4 + b_4)  (seconds), floored by the caller's t_floor.
// Trained on converged plans with the mean squared error of t and Adam; BF16 weights and
// activations in the products, FP32 accumulation, FP32 master weights.  The paper has no
// learned component: this is the warm-start extension of its batched solve.
//
// Kernels (all products on the fifth-generation tensor cores: tcgen05.mma with BF16 operands
// in shared memory, FP32 accumulators in TMEM; weights copied into shared memory by the TMA unit):
//   k_mlp_infer_tc          inference, persistent grid, three 128-row tiles in flight per CTA;
//                           bias + GELU epilogues write the next layer's BF16 operand
//   k_mlp_train_tc          training forward and backward of 128-row tiles: z_l kept in TMEM,
//                           dz_3 -> dh_2 = dz_3 W_3^T -> dz_2 -> dh_1 = dz_2 W_2^T -> dz_1;
//                           writes the layer inputs H_0..H_3, do and dZ_1..dZ_3 feature-major
//   k_mlp_dw_tc             weight gradients dW_l = H_{l-1}^T dZ_l (with the bias gradient from a
//                           row of ones), dw_4 = H_3^T do: M = 128 features, K = rows in 64-row
//                           blocks through a TMA ring, split over row ranges, per-CTA partials
//   k_mlp_dw_reduce, k_mlp_reduce   fixed-order sums of the per-CTA partials into the gradient
//   k_mlp_adam              Adam on the FP32 master weights; k_mlp_pack the BF16 images
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

namespace gmco {
bool tc_encode_map(CUtensorMap *m, const void *ptr, uint64_t cols, uint64_t rows, uint32_t box_cols,
                   uint32_t box_rows);
}

namespace {

constexpr int NIN = 14, NFEAT = 10, NW = 4, KIN = 16, HID = 128;
// flat FP32 parameter layout (the C ABI's): W1 [14][128], b1, W2 [128][128], b2, W3, b3, w4, b4
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NIN * HID, OFF_W2 = OFF_B1 + HID,
              OFF_B2 = OFF_W2 + HID * HID, OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID * HID,
              OFF_W4 = OFF_B3 + HID, OFF_B4 = OFF_W4 + HID, NPARAM = OFF_B4 + 1;
static_assert(NPARAM == GMCO_MLP_NPARAM, "parameter count");
constexpr int MAX_CTAS = 148;

// BF16 weights as the kernels read them.
struct DevWeights {
    float *bias;               // b1, b2, b3, w4 (4 x 128) and b4
    uint8_t *img;              // shared-memory image of W1^T, W2^T, W3^T (forward products)
    uint8_t *imgb;             // shared-memory image of W3, W2 as [k][n] (backward products)
};

// Rows of one call: dense (row = plan * n_dwell + dwell) or listed (pairs[row] = (feature
// row, weight row)).
struct RowSrc {
    const float *feat;      // [n_feat][10]
    const float *w;         // [n_w][4] raw penalty weights
    const int32_t *pairs;   // [R][2] or null (dense)
    int64_t n_feat, n_w;    // listed mode: rows of feat and w (the pairs are checked against them)
    int64_t n_dwell;        // dense mode
    int64_t R;
    const float *target;    // [R] (training)
};

struct TrainOut {
    __nv_bfloat16 *H0, *H1, *H2;      // [16][Rp], [128][Rp], [128][Rp]  layer inputs
    __nv_bfloat16 *dZ1, *dZ2, *dZ3;   // [128][Rp]                      pre-activation grads
    __nv_bfloat16 *H3, *DO, *ONES;    // [128][Rp] GELU(z_3); [16][Rp] row 0 = do; [16][Rp] row 0 = 1
    int64_t Rp;                       // row stride (R rounded up to 128)
    float *part;                      // [gridDim][2]: sum of squared errors, db_4
    float inv_R;                      // 1 / R (mean squared error)
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_d(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
           z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ float softplus(float o) { return o > 20.0f ? o : log1pf(expf(o)); }
__device__ __forceinline__ float sigmoid(float o) { return 1.0f / (1.0f + expf(-o)); }

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
constexpr int32_t kErrPair = 16;                              // status: a pair index out of range

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

// ------------------------------------------------------------------ tcgen05 training
// Backward operand image: W3 and W2 as [k][n] (row k, K = n), the B operand of dh = dz W^T.
constexpr uint32_t IMGB_W3 = 0, IMGB_W2 = 2 * BLK, IMGB_BYTES = 4 * BLK;
constexpr size_t TR_SMEM = IMG_BYTES + IMGB_BYTES + 2 * BLK + 1024;   // weights, one tile, align
constexpr int TR_THREADS = 128;
constexpr uint32_t TR_C0 = 0, TR_C1 = 128, TR_C2 = 256, TR_C3 = 384;   // TMEM column regions

// Feature-major BF16 store of one row's value of feature c: out[c][r].
__device__ __forceinline__ void fm_store(__nv_bfloat16 *out, int64_t ld, int c, int64_t r, float v)
{
    out[(size_t)c * ld + r] = __float2bfloat16_rn(v);
}

// One MMA phase of the training kernel: the tile's operand writes are fenced for the tensor
// core, the group barrier also tells whether any thread's previous wait ran out, the first
// warp issues the layer's products (K = 16 from the first block, or 128 from both) into TMEM
// column region d, and every thread waits for their completion.  Returns false when the
// kernel must stop (uniform over the CTA).
__device__ __forceinline__ bool tr_phase(uint32_t d, uint32_t a_s, uint32_t b_s, bool k16_only, int warp,
                                         uint32_t bar, uint32_t &parity, bool &pending, int32_t *err)
{
    using namespace gmco;
    fence_proxy_async_smem();
    fence_before();
    if (bar_any(1, TR_THREADS, pending)) return false;
    if (warp == 0) {
        fence_after();
        const uint32_t idesc = idesc_bf16(HID);
        if (k16_only) {
            mma_bf16_elect(d, DESC_FIXED | desc_lo(a_s), DESC_FIXED | desc_lo(b_s), idesc, 0u);
        } else {
#pragma unroll
            for (int k = 0; k < HID / 16; ++k) {
                const uint32_t off = (uint32_t)(k >> 2) * BLK + (uint32_t)(k & 3) * 32;
                mma_bf16_elect(d, DESC_FIXED | desc_lo(a_s + off), DESC_FIXED | desc_lo(b_s + off), idesc,
                               k > 0 ? 1u : 0u);
            }
        }
        mma_commit_elect(bar);
    }
    pending = !mbar_wait(bar, parity, err, 2, kMlpWaitNs);
    parity ^= 1u;
    fence_after();
    return true;
}

// Training forward and backward of 128-row tiles on the fifth-generation tensor cores, one
// thread per row (= TMEM lane).  Per tile: the three forward layers (z_l kept in TMEM regions
// C0..C2, FP32), the output unit, the loss and do = dL/do, then dz_3 = do w_4 GELU'(z_3),
// dh_2 = dz_3 W_3^T (region C3), dz_2 = dh_2 GELU'(z_2), dh_1 = dz_2 W_2^T (region C2, z_3 no
// longer needed), dz_1 = dh_1 GELU'(z_1).  The BF16 activations of the next product go
// through the tile's shared-memory blocks; the layer inputs H_0..H_3, do and dZ_1..dZ_3 are
// written feature-major for the weight-gradient GEMMs (H_0's column 14 holds 1, so that the
// bias gradient b_1 comes out of the same product).  Per-CTA partials: the sum of squared
// errors and of do (db_4).
__global__ void __launch_bounds__(TR_THREADS, 1)
    k_mlp_train_tc(const uint8_t *__restrict__ img, const uint8_t *__restrict__ imgb,
                   const float *__restrict__ bias, RowSrc src, TrainOut tr, int32_t *__restrict__ err)
{
    using namespace gmco;
    extern __shared__ uint8_t dyn[];
    __shared__ float sb[4 * HID + 1];
    __shared__ float red[2][TR_THREADS / 32];
    __shared__ __align__(8) uint64_t w_bar, mma_bar, drain_bar;
    __shared__ uint32_t tmem_holder;
    uint8_t *base = reinterpret_cast<uint8_t *>(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t row = (uint32_t)tid;
    const uint32_t s_img = smem_u32(base), s_imgb = s_img + IMG_BYTES;
    uint8_t *sH = base + IMG_BYTES + IMGB_BYTES;
    const uint32_t s_h = smem_u32(sH);
    if (tid == 0) {
        mbar_init(smem_u32(&w_bar), 1);
        mbar_init(smem_u32(&mma_bar), 1);
        mbar_init(smem_u32(&drain_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_holder), 512);
    for (int i = tid; i < 4 * HID + 1; i += TR_THREADS) sb[i] = bias[i];
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_holder;
    if (tid == 0) {
        mbar_expect_tx(smem_u32(&w_bar), IMG_BYTES + IMGB_BYTES);
        for (uint32_t c = 0; c < IMG_BYTES / BLK; ++c) bulk_load(s_img + c * BLK, img + c * BLK, BLK, smem_u32(&w_bar));
        for (uint32_t c = 0; c < IMGB_BYTES / BLK; ++c) bulk_load(s_imgb + c * BLK, imgb + c * BLK, BLK, smem_u32(&w_bar));
    }
    const bool w_ok = mbar_wait(smem_u32(&w_bar), 0u, err, 1, kMlpWaitNs);
    const bool w_fail = __syncthreads_or(!w_ok);
    if (w_fail && tid == 0) mbar_wait(smem_u32(&w_bar), 0u, nullptr, 0, kMlpWaitNs);

    const uint32_t t_lane = tmem + ((uint32_t)(32 * warp) << 16);
    const float *b1 = sb, *b2 = sb + HID, *b3 = sb + 2 * HID, *w4 = sb + 3 * HID;
    const float b4 = sb[4 * HID];
    const uint32_t bar = smem_u32(&mma_bar);
    const int64_t n_tiles = (src.R + 127) / 128, ld = tr.Rp;
    uint32_t parity = 0;
    bool pending = false, failed = w_fail;
    float loss = 0.0f, db4 = 0.0f;
    for (int64_t tile = blockIdx.x; !failed && tile < n_tiles; tile += gridDim.x) {
        const int64_t r = tile * 128 + row;
        bool valid = r < src.R;
        // ---- inputs: BF16 into the tile's first block; H_0 (with the ones column 14)
        {
            float x[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) x[c] = 0.0f;
            int64_t fr = 0, wr = 0;
            if (valid) {
                if (src.pairs) {
                    fr = src.pairs[2 * r];
                    wr = src.pairs[2 * r + 1];
                    if (fr < 0 || fr >= src.n_feat || wr < 0 || wr >= src.n_w) {
                        atomicExch(err, kErrPair);   // a bad pair: the row reads as zeros
                        valid = false;
                    }
                } else {
                    fr = r % src.n_dwell;
                    wr = r / src.n_dwell;
                }
            }
            if (valid) {
#pragma unroll
                for (int c = 0; c < NFEAT; ++c) x[c] = src.feat[fr * NFEAT + c];
#pragma unroll
                for (int c = 0; c < NW; ++c) x[NFEAT + c] = log10f(fmaxf(src.w[wr * NW + c], 1e-3f));
            }
            uint4 lo, hi;
            lo.x = pack_bf16(x[0], x[1]);   lo.y = pack_bf16(x[2], x[3]);
            lo.z = pack_bf16(x[4], x[5]);   lo.w = pack_bf16(x[6], x[7]);
            hi.x = pack_bf16(x[8], x[9]);   hi.y = pack_bf16(x[10], x[11]);
            hi.z = pack_bf16(x[12], x[13]); hi.w = pack_bf16(x[14], x[15]);
            *reinterpret_cast<uint4 *>(sH + swz(row, 0)) = lo;
            *reinterpret_cast<uint4 *>(sH + swz(row, 8)) = hi;
#pragma unroll
            for (int c = 0; c < 16; ++c) fm_store(tr.H0, ld, c, r, c == 14 ? 1.0f : x[c]);
        }
        // ---- forward
        if (!tr_phase(tmem + TR_C0, s_h, s_img + IMG_W1, true, warp, bar, parity, pending, err)) { failed = true; break; }
#pragma unroll 1
        for (int l = 0; l < 2; ++l) {
            const uint32_t cz = l == 0 ? TR_C0 : TR_C1;
            const float *bl = l == 0 ? b1 : b2;
            __nv_bfloat16 *Hout = l == 0 ? tr.H1 : tr.H2;
#pragma unroll 1
            for (int c0 = 0; c0 < HID; c0 += 32) {
                uint32_t v[2][16];
                tmem_ld16(t_lane + cz + (uint32_t)c0, v[0]);
                tmem_ld16(t_lane + cz + (uint32_t)c0 + 16, v[1]);
                tmem_ld_wait16(v[0]);
                tmem_ld_wait16(v[1]);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t h[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int c = 8 * q + 2 * e;
                        const float h0 = gelu(__uint_as_float(v[c >> 4][c & 15]) + bl[c0 + c]);
                        const float h1 = gelu(__uint_as_float(v[c >> 4][(c & 15) + 1]) + bl[c0 + c + 1]);
                        h[e] = pack_bf16(h0, h1);
                        fm_store(Hout, ld, c0 + c, r, h0);
                        fm_store(Hout, ld, c0 + c + 1, r, h1);
                    }
                    *reinterpret_cast<uint4 *>(sH + swz(row, (uint32_t)(c0 + 8 * q))) = make_uint4(h[0], h[1], h[2], h[3]);
                }
            }
            if (!tr_phase(tmem + (l == 0 ? TR_C1 : TR_C2), s_h, s_img + (l == 0 ? IMG_W2 : IMG_W3), false, warp, bar,
                          parity, pending, err)) { failed = true; break; }
        }
        if (failed) break;
        // ---- output unit, loss, do
        float o = 0.0f;
#pragma unroll 1
        for (int c0 = 0; c0 < HID; c0 += 32) {
            uint32_t v[2][16];
            tmem_ld16(t_lane + TR_C2 + (uint32_t)c0, v[0]);
            tmem_ld16(t_lane + TR_C2 + (uint32_t)c0 + 16, v[1]);
            tmem_ld_wait16(v[0]);
            tmem_ld_wait16(v[1]);
#pragma unroll
            for (int c = 0; c < 32; ++c) o = fmaf(gelu(__uint_as_float(v[c >> 4][c & 15]) + b3[c0 + c]), w4[c0 + c], o);
        }
        o += b4;
        const float e = valid ? softplus(o) - src.target[r] : 0.0f;
        const float d_o = valid ? 2.0f * tr.inv_R * e * sigmoid(o) : 0.0f;
        loss += e * e;
        db4 += d_o;
        fm_store(tr.DO, ld, 0, r, d_o);
        // ---- dz_3 = do w_4 GELU'(z_3); H_3 = GELU(z_3) for dw_4
#pragma unroll 1
        for (int c0 = 0; c0 < HID; c0 += 32) {
            uint32_t v[2][16];
            tmem_ld16(t_lane + TR_C2 + (uint32_t)c0, v[0]);
            tmem_ld16(t_lane + TR_C2 + (uint32_t)c0 + 16, v[1]);
            tmem_ld_wait16(v[0]);
            tmem_ld_wait16(v[1]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t h[4];
#pragma unroll
                for (int e2 = 0; e2 < 4; ++e2) {
                    const int c = 8 * q + 2 * e2;
                    float dz[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const float z = __uint_as_float(v[(c + u) >> 4][(c + u) & 15]) + b3[c0 + c + u];
                        fm_store(tr.H3, ld, c0 + c + u, r, gelu(z));
                        dz[u] = d_o * w4[c0 + c + u] * gelu_d(z);
                        fm_store(tr.dZ3, ld, c0 + c + u, r, dz[u]);
                    }
                    h[e2] = pack_bf16(dz[0], dz[1]);
                }
                *reinterpret_cast<uint4 *>(sH + swz(row, (uint32_t)(c0 + 8 * q))) = make_uint4(h[0], h[1], h[2], h[3]);
            }
        }
        // ---- dh_2 = dz_3 W_3^T, dz_2 = dh_2 GELU'(z_2); dh_1 = dz_2 W_2^T, dz_1 = dh_1 GELU'(z_1)
#pragma unroll 1
        for (int l = 0; l < 2; ++l) {
            const uint32_t cd = l == 0 ? TR_C3 : TR_C2;   // dh_2, then dh_1
            const uint32_t cz = l == 0 ? TR_C1 : TR_C0;   // z_2, then z_1
            const float *bl = l == 0 ? b2 : b1;
            __nv_bfloat16 *dZout = l == 0 ? tr.dZ2 : tr.dZ1;
            if (!tr_phase(tmem + cd, s_h, s_imgb + (l == 0 ? IMGB_W3 : IMGB_W2), false, warp, bar, parity, pending,
                          err)) { failed = true; break; }
#pragma unroll 1
            for (int c0 = 0; c0 < HID; c0 += 32) {
                uint32_t dv[2][16], zv[2][16];
                tmem_ld16(t_lane + cd + (uint32_t)c0, dv[0]);
                tmem_ld16(t_lane + cd + (uint32_t)c0 + 16, dv[1]);
                tmem_ld16(t_lane + cz + (uint32_t)c0, zv[0]);
                tmem_ld16(t_lane + cz + (uint32_t)c0 + 16, zv[1]);
                tmem_ld_wait16(dv[0]);
                tmem_ld_wait16(dv[1]);
                tmem_ld_wait16(zv[0]);
                tmem_ld_wait16(zv[1]);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t h[4];
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2) {
                        const int c = 8 * q + 2 * e2;
                        float dz[2];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int cc = c + u;
                            dz[u] = __uint_as_float(dv[cc >> 4][cc & 15]) *
                                    gelu_d(__uint_as_float(zv[cc >> 4][cc & 15]) + bl[c0 + cc]);
                            fm_store(dZout, ld, c0 + cc, r, dz[u]);
                        }
                        h[e2] = pack_bf16(dz[0], dz[1]);
                    }
                    if (l == 0)
                        *reinterpret_cast<uint4 *>(sH + swz(row, (uint32_t)(c0 + 8 * q))) = make_uint4(h[0], h[1], h[2], h[3]);
                }
            }
        }
    }
    // per-CTA partials in a fixed order: warp sums, then the warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        loss += __shfl_xor_sync(0xffffffffu, loss, o);
        db4 += __shfl_xor_sync(0xffffffffu, db4, o);
    }
    if (lane == 0) {
        red[0][warp] = loss;
        red[1][warp] = db4;
    }
    fence_before();
    if (!failed) failed = bar_any(1, TR_THREADS, pending);
    if (failed && !w_fail && warp == 0) {
        mma_commit_elect(smem_u32(&drain_bar));
        mbar_wait(smem_u32(&drain_bar), 0u, nullptr, 0, kMlpWaitNs);
    }
    fence_before();
    __syncthreads();
    if (tid == 0) {
        float sl = 0.0f, sd = 0.0f;
        for (int w = 0; w < TR_THREADS / 32; ++w) {
            sl += red[0][w];
            sd += red[1][w];
        }
        tr.part[(size_t)blockIdx.x * 2 + 0] = sl;
        tr.part[(size_t)blockIdx.x * 2 + 1] = sd;
    }
    if (warp == 0) {
        fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// Weight-gradient GEMM on the tensor cores: D[m][j] = sum over the CTA's rows r of A[m][r] B[j][r]
// (A 128 features, B N_b rows, plus N_2 rows from a second map when n_2 > 0, all feature-major
// BF16 with rows r contiguous), M = 128, N = N_b + n_2, K = rows in blocks of 64 through a
// four-stage ring: a producer thread (warp 0), an MMA thread (warp 1), the accumulator read
// back by all four warps into the CTA's FP32 partial part[cta][128][N].
constexpr int DW_STAGES = 4;
constexpr uint32_t DW_A = 0, DW_B = BLK, DW_B2 = 2 * BLK, DW_STAGE = 2 * BLK + 2048;   // 34 KB
constexpr size_t DW_SMEM = (size_t)DW_STAGES * DW_STAGE + 1024;

__global__ void __launch_bounds__(128, 1)
    k_mlp_dw_tc(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap mb,
                const __grid_constant__ CUtensorMap mb2, int32_t n_b, int32_t n_2, int64_t kb_total,
                int64_t kb_chunk, float *__restrict__ part, int32_t *__restrict__ err)
{
    using namespace gmco;
    extern __shared__ uint8_t dyn[];
    __shared__ __align__(8) uint64_t full_bar[DW_STAGES], empty_bar[DW_STAGES], done_bar;
    __shared__ uint32_t tmem_holder;
    uint8_t *base = reinterpret_cast<uint8_t *>(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
    const uint32_t s0 = smem_u32(base);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = n_b + n_2;
    const int64_t kb0 = blockIdx.x * kb_chunk, kb1 = min(kb0 + kb_chunk, kb_total);
    if (tid == 0) {
        for (int s = 0; s < DW_STAGES; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&done_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_holder), 256);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_holder;
    __shared__ int s_fail;
    if (tid == 0) s_fail = 0;
    __syncthreads();
    int armed = 0;   // producer: stages armed, for the wind-down
    if (warp == 0 && lane == 0) {
        const uint32_t bytes = (uint32_t)(BLK + n_b * 128 + n_2 * 128);
        for (int64_t kb = kb0; kb < kb1; ++kb, ++armed) {
            const int it = (int)(kb - kb0), s = it % DW_STAGES;
            const uint32_t ph = (uint32_t)(it / DW_STAGES) & 1u;
            if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, err, 1, kMlpWaitNs)) { s_fail = 1; break; }
            const uint32_t st = s0 + (uint32_t)s * DW_STAGE, fb = smem_u32(&full_bar[s]);
            mbar_expect_tx(fb, bytes);
            tma_load_2d(st + DW_A, &ma, (int)(kb * 64), 0, fb);
            tma_load_2d(st + DW_B, &mb, (int)(kb * 64), 0, fb);
            if (n_2 > 0) tma_load_2d(st + DW_B2, &mb2, (int)(kb * 64), 0, fb);
        }
    } else if (warp == 1) {
        const uint32_t idesc = idesc_bf16(N);
        bool ok = true;
        for (int64_t kb = kb0; kb < kb1 && ok; ++kb) {
            const int it = (int)(kb - kb0), s = it % DW_STAGES;
            const uint32_t ph = (uint32_t)(it / DW_STAGES) & 1u;
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&full_bar[s]), ph, err, 2, kMlpWaitNs))) {
                ok = false;
                break;
            }
            fence_after();
            const uint32_t st = s0 + (uint32_t)s * DW_STAGE;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mma_bf16_elect(tmem, DESC_FIXED | desc_lo(st + DW_A + 32u * k), DESC_FIXED | desc_lo(st + DW_B + 32u * k),
                               idesc, (kb == kb0 && k == 0) ? 0u : 1u);
            mma_commit_elect(smem_u32(&empty_bar[s]));
        }
        if (!ok && lane == 0) s_fail = 1;
        mma_commit_elect(smem_u32(&done_bar));   // completes once every MMA issued has finished
    }
    const bool done = mbar_wait(smem_u32(&done_bar), 0u, err, 3, kMlpWaitNs);
    if (!done) {
        if (tid == 0) s_fail = 1;
        mbar_wait(smem_u32(&done_bar), 0u, nullptr, 0, kMlpWaitNs);
    }
    fence_after();
    __syncthreads();
    if (warp == 0 && lane == 0 && s_fail) {
        // copies this thread armed may still be landing: wait (bounded) for their phases
        for (int s = 0; s < DW_STAGES; ++s) {
            if (armed <= s) continue;
            const int last = armed - 1 - ((armed - 1 - s) % DW_STAGES);
            mbar_wait(smem_u32(&full_bar[s]), (uint32_t)(last / DW_STAGES) & 1u, nullptr, 0, kMlpWaitNs);
        }
    }
    if (!s_fail && kb1 > kb0) {
        const int m = 32 * warp + lane;
        float *out = part + ((size_t)blockIdx.x * 128 + m) * N;
        for (int c = 0; c < N; c += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
            tmem_ld_wait16(v);
#pragma unroll
            for (int j = 0; j < 16; ++j) out[c + j] = __uint_as_float(v[j]);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        tmem_dealloc(tmem, 256);
    }
}

// grad[dst + j * sj + m * sm] = sum over CTAs c < n (in order) of part[c][m][j0 + j], for
// m < 128 and j < nj (N columns per partial row).
__global__ void k_mlp_dw_reduce(const float *__restrict__ part, int32_t n, int32_t N, int32_t j0, int32_t nj,
                                float *__restrict__ grad, int64_t dst, int64_t sj, int64_t sm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 128 * nj) return;
    const int m = i % 128, j = i / 128;
    float s = 0.0f;
    for (int c = 0; c < n; ++c) s += part[((size_t)c * 128 + m) * N + j0 + j];
    grad[dst + j * sj + m * sm] = s;
}

// BF16 copies of the FP32 master parameters in the kernels' layouts.
__global__ void k_mlp_pack(const float *__restrict__ p, DevWeights w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < HID * 64) {
        const int n = i / 64, k = i % 64;     // one 64-column block of W1^T, columns 14.. zero
        img_put(w.img, IMG_W1, n, k, k < NIN ? p[OFF_W1 + k * HID + n] : 0.0f);
    }
    if (i < HID * HID) {
        const int k = i / HID, n = i % HID;
        img_put(w.img, IMG_W2, n, k, p[OFF_W2 + i]);
        img_put(w.img, IMG_W3, n, k, p[OFF_W3 + i]);
        img_put(w.imgb, IMGB_W2, k, n, p[OFF_W2 + i]);
        img_put(w.imgb, IMGB_W3, k, n, p[OFF_W3 + i]);
    }
    if (i < 4 * HID + 1) {
        // bias[] = b1, b2, b3, w4 (128 each), then b4
        const int blk = i / HID, o = i % HID;
        const int srcs[4] = {OFF_B1, OFF_B2, OFF_B3, OFF_W4};
        w.bias[i] = i == 4 * HID ? p[OFF_B4] : p[srcs[blk] + o];
    }
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

__global__ void k_mlp_fill_ones(__nv_bfloat16 *ones, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) ones[i] = __float2bfloat16_rn(1.0f);
}

// Loss and gradient (into q->grad) of the batch at the current BF16 weights, on the tensor
// cores: k_mlp_train_tc for the forward and backward of every row, four weight-gradient GEMMs
// (W_1 with b_1, W_2 with b_2, W_3 with b_3, w_4) and fixed-order reductions of the per-CTA
// partials.
gmco_status gradient_tc(gmco_mlp *q, const RowSrc &src, float *loss_out)
{
    const int64_t R = src.R;
    const int64_t Rp = (R + 127) / 128 * 128;
    if (Rp > q->cap_rows) {
        MCK(cudaStreamSynchronize(q->stream));
        free_ws(q);
        TrainOut &t = q->tr;
        MCK(dalloc(q, &t.H0, (size_t)KIN * Rp, true));
        MCK(dalloc(q, &t.H1, (size_t)HID * Rp, true));
        MCK(dalloc(q, &t.H2, (size_t)HID * Rp, true));
        MCK(dalloc(q, &t.H3, (size_t)HID * Rp, true));
        MCK(dalloc(q, &t.dZ1, (size_t)HID * Rp, true));
        MCK(dalloc(q, &t.dZ2, (size_t)HID * Rp, true));
        MCK(dalloc(q, &t.dZ3, (size_t)HID * Rp, true));
        MCK(dalloc(q, &t.DO, (size_t)16 * Rp, true));
        MCK(dalloc(q, &t.ONES, (size_t)16 * Rp, true));
        MCK(dalloc(q, &t.part, (size_t)MAX_CTAS * 2, true));
        MCK(dalloc(q, &q->dwpart, (size_t)MAX_CTAS * 128 * 144, true));
        // rows 1..15 of DO and ONES stay zero; row 0 of ONES is one
        MCK(cudaMemsetAsync(t.DO, 0, (size_t)16 * Rp * sizeof(__nv_bfloat16), q->stream));
        MCK(cudaMemsetAsync(t.ONES, 0, (size_t)16 * Rp * sizeof(__nv_bfloat16), q->stream));
        k_mlp_fill_ones<<<(unsigned)((Rp + 255) / 256), 256, 0, q->stream>>>(t.ONES, Rp);
        MCK(cudaGetLastError());
        q->cap_rows = Rp;
    }
    TrainOut tr = q->tr;
    tr.Rp = Rp;
    tr.inv_R = 1.0f / (float)R;
    int n_sm = 0;
    MCK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, q->device));
    const int ctas = (int)std::min<int64_t>(std::min(n_sm, MAX_CTAS), Rp / 128);
    MCK(cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TR_SMEM));
    k_mlp_train_tc<<<ctas, TR_THREADS, TR_SMEM, q->stream>>>(q->w.img, q->w.imgb, q->w.bias, src, tr, q->err);
    MCK(cudaGetLastError());
    q->launches++;
    // weight gradients: D = A B^T over row ranges of 64-row blocks
    const int64_t kb_total = Rp / 64;
    const int64_t kb_chunk = std::max<int64_t>(4, (kb_total + n_sm - 1) / n_sm);
    const int n_dw = (int)((kb_total + kb_chunk - 1) / kb_chunk);   // every CTA has a block
    struct Job {
        const __nv_bfloat16 *A, *B, *B2;
        int n_b, n_2;
        int64_t w_off, b_off;   // weight block (j = k < nk) and bias column (j = n_b), -1: none
        int nk;
    };
    const Job jobs[4] = {
        {tr.dZ1, tr.H0, nullptr, 16, 0, OFF_W1, OFF_B1, NIN},     // column 14 of H0 is one
        {tr.dZ2, tr.H1, tr.ONES, 128, 16, OFF_W2, OFF_B2, HID},
        {tr.dZ3, tr.H2, tr.ONES, 128, 16, OFF_W3, OFF_B3, HID},
        {tr.H3, tr.DO, nullptr, 16, 0, OFF_W4, -1, 1},
    };
    MCK(cudaFuncSetAttribute(k_mlp_dw_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DW_SMEM));
    const int rb = 256;
    for (const Job &jb : jobs) {
        CUtensorMap ma, mb, mb2;
        if (!gmco::tc_encode_map(&ma, jb.A, (uint64_t)Rp, 128, 64, 128) ||
            !gmco::tc_encode_map(&mb, jb.B, (uint64_t)Rp, (uint64_t)jb.n_b, 64, (uint32_t)jb.n_b) ||
            !gmco::tc_encode_map(&mb2, jb.B2 ? jb.B2 : jb.B, (uint64_t)Rp, 16, 64, 16)) {
            g_mlp_err = "gradient: tensor map encoding failed";
            return GMCO_ECUDA;
        }
        const int N = jb.n_b + jb.n_2;
        k_mlp_dw_tc<<<n_dw, 128, DW_SMEM, q->stream>>>(ma, mb, mb2, jb.n_b, jb.n_2, kb_total, kb_chunk, q->dwpart, q->err);
        MCK(cudaGetLastError());
        // D[m = n][j = k]: the weight W[k][n] at w_off + k * 128 + n (for w_4: w_off + n)
        const int64_t sj = jb.nk == 1 ? 0 : HID;
        k_mlp_dw_reduce<<<(unsigned)((128 * jb.nk + rb - 1) / rb), rb, 0, q->stream>>>(q->dwpart, n_dw, N, 0, jb.nk,
                                                                                     q->grad, jb.w_off, sj, 1);
        q->launches += 2;
        if (jb.b_off >= 0) {
            const int jb_col = jb.n_2 > 0 ? jb.n_b : 14;   // the ones row: ONES row 0, or H0 column 14
            k_mlp_dw_reduce<<<1, 128, 0, q->stream>>>(q->dwpart, n_dw, N, jb_col, 1, q->grad, jb.b_off, 0, 1);
            q->launches++;
        }
        MCK(cudaGetLastError());
    }
    // db_4 and the loss from the per-CTA partials (loss, db_4)
    k_mlp_reduce<<<1, 32, 0, q->stream>>>(tr.part, ctas, 2, 1, 1, q->grad, OFF_B4);
    k_mlp_reduce<<<1, 32, 0, q->stream>>>(tr.part, ctas, 2, 0, 1, q->grad + NPARAM, 0);
    MCK(cudaGetLastError());
    q->launches += 2;
    MCK(cudaMemcpyAsync(q->h_pinned + 1, q->err, sizeof(int32_t), cudaMemcpyDeviceToHost, q->stream));
    if (loss_out) MCK(cudaMemcpyAsync(q->h_pinned, q->grad + NPARAM, sizeof(float), cudaMemcpyDeviceToHost, q->stream));
    MCK(cudaStreamSynchronize(q->stream));
    int32_t code = 0;
    memcpy(&code, q->h_pinned + 1, sizeof code);
    if (code != 0) {
        cudaMemsetAsync(q->err, 0, sizeof(int32_t), q->stream);
        cudaStreamSynchronize(q->stream);
        if (code == kErrPair) {
            g_mlp_err = "pair index out of range";
            return GMCO_EINVAL;
        }
        g_mlp_err = "gradient: a tensor-core wait of the training kernels ran out (code " + std::to_string(code) + ")";
        return GMCO_ECUDA;
    }
    if (loss_out) *loss_out = q->h_pinned[0] / (float)R;
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
    // the training kernel checks every pair against these counts before it reads a row
    // (a row out of range is read as zeros and the call fails with GMCO_EINVAL)
    s.n_feat = n_feat;
    s.n_w = n_w;
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
        dalloc(q, &q->w.bias, 4 * HID + 1) != cudaSuccess ||
        dalloc(q, &q->w.img, IMG_BYTES) != cudaSuccess || dalloc(q, &q->w.imgb, IMGB_BYTES) != cudaSuccess ||
        dalloc(q, &q->err, 1) != cudaSuccess)
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
    if ((r = gradient_tc(q, s, &l)) != GMCO_OK) return r;
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
    if ((r = gradient_tc(q, s, loss ? &l : nullptr)) != GMCO_OK) return r;
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
