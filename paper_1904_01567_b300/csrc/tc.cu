// Tensor-core evaluation of Eq. (dose), Eq. (1), Eq. (obj) and Eq. (2) on sm_103a:
// tcgen05.mma (kind::f16, BF16 operands, FP32 accumulators in TMEM), operands staged by TMA
// (cp.async.bulk.tensor, 128-byte swizzle) through an mbarrier ring, one elected thread
// issuing the MMAs, sixteen epilogue warps (four per TMEM lane quarter) reading TMEM with tcgen05.ld.
//
// A row i of A is scaled by a power of two s_i (exact) and split into BF16 terms
// A/s = A1 + A2 + A3; t and dF/dd are split the same way.  Products A_i T_j are exact in FP32,
// and keeping the pairs with i + j <= n + 1 (n = number of terms) leaves an error of the
// order of the last kept term: 2^-8 relative for one term, 2^-16 for two, 2^-24 for three.
//
// Dose GEMM (rows = plans, columns = points, K = dwells):
//   acc0 = sum_{i,j} T_j A_i^T            -> d = s * acc0
//   acc1 = sum_i dT1 A_i^T + dT2 A_1^T    -> dd = s * acc1, the dose change of the step
//   (dT = dT1 + dT2 in two BF16 terms: the objective change sums f(d) - f(d - dd) over points
//   whose first-order parts nearly cancel near the optimum, so a 2^-9 relative error in dd
//   would swamp the Armijo and stop tests there)
//   epilogue: Eq. (1) penalty, per-plan partial of F and of F(t) - F(t - dT) (factored, see
//   eval_simt.cu), and G = s * dF/dd split into BF16 terms for the gradient GEMM.
// Gradient GEMM (rows = plans, columns = dwells, K = points, split over point ranges):
//   acc0 = sum_{i,j} G_j A_i               -> partial of A^T G, reduced by k_finish.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "tc.cuh"
#include "tcgen05.cuh"

namespace gmco {

namespace {

constexpr int BM = 128;                 // M rows per tile (TMEM lanes): points or dwells
constexpr int BK = 64;                  // K elements per stage: 128 bytes of BF16
constexpr int EPI_WARPS = 16;           // 4 per TMEM lane quarter
constexpr int EPI_GROUPS = EPI_WARPS / 4;   // column groups of the epilogue
constexpr int W_TMA = EPI_WARPS, W_MMA = EPI_WARPS + 1, W_TMEM = EPI_WARPS + 2;
constexpr int NTHREADS = (EPI_WARPS + 3) * 32;   // epilogue, TMA, MMA, TMEM owner
constexpr int MAX_STAGES = 4;
constexpr int SMEM_BUDGET = 194 * 1024;   // dynamic ring; with ~32 KB of static shared memory
                                          // the total stays within the 227 KB of a CTA
constexpr int TMEM_COLS = 512;          // two accumulator buffers
constexpr int BUF_COLS = 256;
constexpr long long kDrainNs = 1000000000LL;   // wind-down waits after a failed wait: 1 s

// ------------------------------------------------------------------ the GEMM kernel

// The MMAs of one stage: k16n K steps (16 each) of the group's NP products, all issued by the
// elected lane of the converged MMA warp.  NP is a template parameter so that the loop has no
// per-product predicates.
template <int NP>
__device__ __forceinline__ void issue_stage(uint32_t tbuf, uint32_t st_lo, const uint32_t *aq,
                                            const uint32_t *bq, const uint32_t *iq, int k16n,
                                            bool fresh)
{
#pragma unroll
    for (int k16 = 0; k16 < 4; ++k16) {
        if (k16 < k16n) {
            const uint32_t kk = st_lo + 2u * (uint32_t)k16;
#pragma unroll
            for (int q = 0; q < NP; ++q)
                mma_bf16_elect(tbuf, DESC_FIXED | (kk + aq[q]), DESC_FIXED | (kk + bq[q]), iq[q],
                               (fresh && k16 == 0 && q == 0) ? 0u : 1u);
        }
    }
}

// One kind of ring stage: the M-side tiles (a_map, 128 rows each) and the N-side slots loaded
// for one K block, and the products issued on them.  A slot holds one or two boxes of 128
// rows stacked in shared memory (b_map[slot][0], b_map[slot][1]; -1 = none; b_roff = row
// offset of a box), so that one MMA of N = 256 multiplies an M-side tile by both: in the dose
// GEMM a slot is [T_j | dT_j], and one product gives A_i T_j and A_i dT_j side by side; in the
// gradient GEMM it is a 256-plan tile of G_j in two halves.  Product q multiplies tile
// pair_a[q] by slot pair_b[q] with N = pair_n[q].  Fewer, wider MMAs matter here: the single
// issuing thread shares the SM with the epilogue warps, and its issue rate, not the tensor
// pipe, bounds a stream of N = 128 MMAs (measured).
constexpr int MAX_A = 3, MAX_B = 3, MAX_PAIRS = 8;
constexpr int BOX = BM * BK * 2;        // bytes of one 128-row box of a K block
struct Group {
    int32_t n_a, n_b, n_pair;
    int32_t a_map[MAX_A];
    int32_t b_map[MAX_B][2], b_roff[MAX_B][2];
    int32_t pair_a[MAX_PAIRS], pair_b[MAX_PAIRS], pair_n[MAX_PAIRS];
};

// Launch parameters common to every problem of the list.
struct KParams {
    TcMaps maps;
    const void *probs;        // TcDoseProb[n_probs] (dose GEMM) or TcGradProb[n_probs]
    int32_t n_probs, parity;
    int32_t has_dT, write_dose, zero_next;
    int32_t sparse_ok;        // a solver step: the active-set gradient may be chosen
    int32_t nG;               // BF16 terms of G written by the dose epilogue
    int32_t bn;               // plans per tile: 128 (dose GEMM), 256 or 128 (gradient GEMM)
    int32_t n_groups;
    Group g[3];
    int32_t n_stages, stage_bytes, slot_bytes;   // ring stage size, size of one N-side slot
    int32_t b_off;                               // offset of the N-side slots in a stage
    const void *pf_ptr[kTcPrefetch];             // gradient GEMM: L2 prefetch ranges (bytes)
    int64_t pf_bytes[kTcPrefetch];
    int32_t *err;
    int64_t wait_ns;                             // limit of every pipeline wait
};

template <int KIND>
struct ProbOf;
template <>
struct ProbOf<1> { using type = TcDoseProb; };
template <>
struct ProbOf<2> { using type = TcGradProb; };

__device__ __forceinline__ int find_prob(const int32_t *start, int p, int item)
{
    while (item >= start[p + 1]) ++p;   // items are visited in increasing order
    return p;
}

// A work item decoded: plan tile, point tile (dose GEMM) or dwell tile and point split
// (gradient GEMM), and whether a gradient plan tile of 256 holds at most 128 valid rows (its
// products then run with N = 128 on the first half).
struct Item {
    int p, ptile, sub, dt;
    bool half;
};

template <int KIND>
__device__ __forceinline__ Item decode_item(const int32_t *s_start, const int32_t *s_per,
                                            const int32_t *s_nsplit, const int32_t *s_rows, int bn,
                                            int p, int item)
{
    Item it;
    it.p = find_prob(s_start, p, item);
    const int local = item - s_start[it.p];
    it.ptile = local / s_per[it.p];
    const int r = local - it.ptile * s_per[it.p];
    if constexpr (KIND == 1) {
        it.sub = r;
        it.dt = 0;
        it.half = false;
    } else {
        it.dt = r / s_nsplit[it.p];
        it.sub = r - it.dt * s_nsplit[it.p];
        it.half = bn > 128 && s_rows[it.p] - it.ptile * bn <= 128;
    }
    return it;
}

// Column sums over a warp of 8 values per lane, in a fixed order: afterwards every lane holds
// the sum over all 32 lanes of column (lane >> 2) & 7.  Three halving exchanges leave each
// lane one column summed over 8 lanes; two more add the 4 lanes that share it.
__device__ __forceinline__ float warp_col_sum8(const float (&v)[8], int lane)
{
    constexpr unsigned kAll = 0xffffffffu;
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float w[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const float keep = b4 ? v[t + 4] : v[t], give = b4 ? v[t] : v[t + 4];
        w[t] = keep + __shfl_xor_sync(kAll, give, 16);
    }
    float y[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const float keep = b3 ? w[t + 2] : w[t], give = b3 ? w[t] : w[t + 2];
        y[t] = keep + __shfl_xor_sync(kAll, give, 8);
    }
    float z = (b2 ? y[1] : y[0]) + __shfl_xor_sync(kAll, b2 ? y[0] : y[1], 4);
    z += __shfl_xor_sync(kAll, z, 2);
    z += __shfl_xor_sync(kAll, z, 1);
    return z;
}

// 8 x 8 transpose within each group of 8 lanes: lane r of a group holds row r (v[i] = M[r][i])
// before and column r (v[j] = M[j][r]) after.  Three butterfly stages; the one at distance s
// swaps the elements whose row and column differ in bit s.
__device__ __forceinline__ void transpose8(uint32_t (&v)[8], int lane)
{
#pragma unroll
    for (int s = 4; s >= 1; s >>= 1) {
        const bool up = lane & s;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i & s) continue;
            const uint32_t send = up ? v[i] : v[i | s];
            const uint32_t recv = __shfl_xor_sync(0xffffffffu, send, s);
            if (up) v[i] = recv;
            else v[i | s] = recv;
        }
    }
}

constexpr int kClStride = 132;   // row stride of the per-plan weight tables (bank spread)

// Persistent: the grid is at most one CTA per SM, and each CTA walks the work items of all
// problems of the launch (dose GEMM: problem x plan tile x point tile; gradient GEMM:
// problem x plan tile x dwell tile x point split), derived from each problem's compact-row
// count at run time.  The problems' descriptors are staged in shared memory.  The TMA ring
// continues across items; accumulators live in two TMEM buffers of 256 columns handed
// between the MMA thread and the epilogue warps through acc_full / acc_empty barriers, so the
// epilogue of one item overlaps the MMAs of the next.  TMEM lanes are points (dose GEMM) or
// dwells (gradient GEMM); columns are plans.
template <int KIND>   // 1: dose GEMM with penalty epilogue, 2: gradient GEMM
__global__ void __launch_bounds__(NTHREADS, 1) k_tc(const __grid_constant__ KParams kp)
{
    using Prob = typename ProbOf<KIND>::type;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    __shared__ __align__(8) uint64_t full_bar[MAX_STAGES], empty_bar[MAX_STAGES];
    __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2];
    __shared__ __align__(8) uint64_t drain_bar;   // MMA completion after a failed wait
    __shared__ int32_t s_wound;                   // some role of this CTA gave up a wait
    __shared__ int32_t s_prod_it;                 // ring stages the producer armed
    __shared__ uint32_t tmem_holder;
    __shared__ __align__(16) Prob s_prob[kMaxMulti];
    __shared__ int32_t s_start[kMaxMulti + 1];   // first work item of each problem
    __shared__ int32_t s_rows[kMaxMulti];        // compact rows of each problem
    __shared__ int32_t s_per[kMaxMulti];         // work items per plan tile
    __shared__ int32_t s_kbps[kMaxMulti];        // gradient GEMM: K blocks per split
    __shared__ int32_t s_nsplit[kMaxMulti];      // gradient GEMM: splits
    __shared__ int32_t s_sparse[kMaxMulti];      // dose GEMM: this step's path is the active-set gradient
    __shared__ int32_t s_fail;
    __shared__ int32_t s_act;                    // dose GEMM: active (plan, point) pairs of this CTA
    __shared__ __align__(16) float s_cl[8][kClStride], s_ch[8][kClStride];   // w/N w_min, w/N w_max per plan
    __shared__ float s_part[2][4][BM];           // per lane quarter and plan: partial F, dF
    __shared__ __align__(16) uint16_t s_gst[KIND == 1 ? EPI_WARPS : 1][8 * 32];   // dose GEMM: G staging per warp

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int np = kp.n_probs;
    const Prob *gprob = static_cast<const Prob *>(kp.probs);
    {
        static_assert(sizeof(Prob) % 4 == 0, "descriptor size");
        const uint32_t *src = reinterpret_cast<const uint32_t *>(gprob);
        uint32_t *dst = reinterpret_cast<uint32_t *>(s_prob);
        const int words = np * (int)(sizeof(Prob) / 4);
        for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    }
    if ((int)threadIdx.x < np) {
        const int p = threadIdx.x;
        const Prob &d = gprob[p];
        const int rows = *d.n_rows[kp.parity];
        int per = 1, kbps = 0, nsplit = 1, rows_run = rows;
        if constexpr (KIND == 1) {
            per = d.n_ptiles;
            if (kp.zero_next && blockIdx.x == 0) *const_cast<int32_t *>(d.n_rows[kp.parity ^ 1]) = 0;
            // path of this step, from the previous step's active-pair count (every CTA decides
            // alike; CTA 0 records it for the gradient kernels and the update)
            int sparse = 0;
            if (d.act) {
                sparse = kp.sparse_ok && (int64_t)d.act[kp.parity ^ 1] <= (int64_t)d.sp_thr * rows ? 1 : 0;
                if (blockIdx.x == 0) d.act[2 + kp.parity] = sparse;
            }
            s_sparse[p] = sparse;
        } else {
            split_plan(d.sp, rows, &kbps, &nsplit);
            per = d.n_dt * nsplit;
            if (d.act && d.act[2 + kp.parity]) rows_run = 0;   // the active-set gradient serves this step
        }
        s_rows[p] = rows_run;
        s_per[p] = per;
        s_kbps[p] = kbps;
        s_nsplit[p] = nsplit;
    }
    if (threadIdx.x == 0) {
        s_fail = 0;
        s_act = 0;
        s_wound = 0;
        s_prod_it = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int p = 0; p < np; ++p) {
            s_start[p] = acc;
            acc += ((s_rows[p] + kp.bn - 1) / kp.bn) * s_per[p];
        }
        s_start[np] = acc;
    }
    __syncthreads();
    const int n_items = s_start[np];
    if ((int)blockIdx.x >= n_items) return;   // no work: leave before any barrier or TMEM use

    if (threadIdx.x == 0) {
        for (int s = 0; s < kp.n_stages; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&accf_bar[b]), 1);
            mbar_init(smem_u32(&acce_bar[b]), EPI_WARPS);   // one arrival per epilogue warp
        }
        mbar_init(smem_u32(&drain_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == W_TMEM) tmem_alloc(smem_u32(&tmem_holder), (uint32_t)TMEM_COLS);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_holder;

    if (warp == W_TMA) {
        // ---------------- TMA producer (one thread)
        if (lane == 0) {
            int it = 0, p = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
                const Item w = decode_item<KIND>(s_start, s_per, s_nsplit, s_rows, kp.bn, p, item);
                p = w.p;
                const Prob &d = s_prob[p];
                int arow, brow, kb0, kb1;
                if constexpr (KIND == 1) {
                    arow = d.a_row + w.sub * BM;
                    brow = d.t_row + w.ptile * kp.bn;
                    kb0 = 0;
                    kb1 = d.kb;
                } else {
                    arow = d.at_row + w.dt * BM;
                    brow = d.g_row + w.ptile * kp.bn;
                    kb0 = w.sub * s_kbps[p];
                    kb1 = min(kb0 + s_kbps[p], d.kb);
                }
                for (int gi = 0; gi < kp.n_groups && ok; ++gi) {
                    const Group &g = kp.g[gi];
                    uint32_t bytes = (uint32_t)(g.n_a * BOX);
                    for (int b = 0; b < g.n_b; ++b)
                        bytes += (uint32_t)BOX * ((g.b_map[b][1] >= 0 && !w.half) ? 2u : 1u);
                    for (int kb = kb0; kb < kb1; ++kb, ++it) {
                        const int s = it % kp.n_stages;
                        const uint32_t ph = (uint32_t)(it / kp.n_stages) & 1u;
                        if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, kp.err, 1, kp.wait_ns)) { ok = false; break; }
                        uint8_t *st = smem + (size_t)s * kp.stage_bytes;
                        const uint32_t fb = smem_u32(&full_bar[s]);
                        mbar_expect_tx(fb, bytes);
                        for (int t = 0; t < g.n_a; ++t)
                            tma_load_2d(smem_u32(st + t * BOX), &kp.maps.m[g.a_map[t]], kb * BK, arow, fb);
                        for (int b = 0; b < g.n_b; ++b) {
                            uint8_t *slot = st + kp.b_off + b * kp.slot_bytes;
                            tma_load_2d(smem_u32(slot), &kp.maps.m[g.b_map[b][0]], kb * BK,
                                        brow + g.b_roff[b][0], fb);
                            if (g.b_map[b][1] >= 0 && !w.half)
                                tma_load_2d(smem_u32(slot + BOX), &kp.maps.m[g.b_map[b][1]], kb * BK,
                                            brow + g.b_roff[b][1], fb);
                        }
                    }
                }
            }
            s_prod_it = it;   // stages armed, for the wind-down after a failed wait
            if (!ok) s_wound = 1;
        }
        if constexpr (KIND == 2) {
            // once this CTA's operand loads are all issued (its MMAs and epilogue still to
            // come), L2 prefetch of the update's operands, in 16 KB pieces shared out over the
            // CTAs that have work
            __syncwarp();
            constexpr int64_t PIECE = 16384;
            const int64_t ctas = min((int64_t)gridDim.x, (int64_t)n_items);
            for (int r = 0; r < kTcPrefetch; ++r) {
                const char *base = static_cast<const char *>(kp.pf_ptr[r]);
                const int64_t bytes = kp.pf_bytes[r];
                const int64_t pieces = (bytes + PIECE - 1) / PIECE;
                for (int64_t c = blockIdx.x + lane * ctas; c < pieces; c += 32 * ctas) {
                    const int64_t off = c * PIECE;
                    prefetch_l2(base + off, (uint32_t)min(PIECE, bytes - off));
                }
            }
        }
    } else if (warp == W_MMA) {
        // ---------------- MMA issuer (the whole warp walks the items; one elected lane issues)
        {
            int p = 0, nb = 0;
            int st_i = 0;            // stage of the ring and the parity of its current use
            uint32_t st_ph = 0u;
            uint32_t use[2] = {0u, 0u};   // completed uses of each accumulator buffer
            bool ok = true;
            const uint32_t s_lo0 = desc_lo(smem_u32(smem));
            const uint32_t stage_lo = (uint32_t)kp.stage_bytes >> 4;
            for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
                const Item w = decode_item<KIND>(s_start, s_per, s_nsplit, s_rows, kp.bn, p, item);
                p = w.p;
                const Prob &d = s_prob[p];
                int kb0, kb1, k16_total;
                if constexpr (KIND == 1) {
                    kb0 = 0;
                    kb1 = d.kb;
                    k16_total = d.k16;
                } else {
                    kb0 = w.sub * s_kbps[p];
                    kb1 = min(kb0 + s_kbps[p], d.kb);
                    k16_total = 1 << 30;
                }
                const int buf = nb;
                if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&acce_bar[buf]), (use[buf] & 1u) ^ 1u, kp.err, 4, kp.wait_ns)))
                    break;
                fence_after();
                const uint32_t tbuf = tmem + (uint32_t)(buf * BUF_COLS);
                for (int gi = 0; gi < kp.n_groups && ok; ++gi) {
                    const Group &g = kp.g[gi];
                    const int npair = g.n_pair;
                    // per product: descriptor address fields (16-byte units) of its tiles
                    // relative to the stage, and its instruction descriptor; in the loop a
                    // descriptor is DESC_FIXED | (stage + offset + 2 per 32-byte K step)
                    uint32_t aq[MAX_PAIRS], bq[MAX_PAIRS], iq[MAX_PAIRS];
#pragma unroll
                    for (int q = 0; q < MAX_PAIRS; ++q) {
                        const int qq = q < npair ? q : 0;
                        aq[q] = (uint32_t)(g.pair_a[qq] * BOX) >> 4;
                        bq[q] = (uint32_t)(kp.b_off + g.pair_b[qq] * kp.slot_bytes) >> 4;
                        iq[q] = idesc_bf16(w.half ? 128 : g.pair_n[qq]);
                    }
                    for (int kb = kb0; kb < kb1; ++kb) {
                        const int s = st_i;
                        const uint32_t ph = st_ph;
                        if (++st_i == kp.n_stages) {
                            st_i = 0;
                            st_ph ^= 1u;
                        }
                        if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&full_bar[s]), ph, kp.err, 2, kp.wait_ns))) {
                            ok = false;   // warp-uniform
                            break;
                        }
                        fence_after();
                        const uint32_t st_lo = s_lo0 + (uint32_t)s * stage_lo;
                        // the first product of the item (an N = 256 one whenever any is)
                        // starts the accumulator
                        const bool fresh = gi == 0 && kb == kb0;
                        const int k16n = min(4, k16_total - kb * 4);
                        switch (npair) {
                        case 1: issue_stage<1>(tbuf, st_lo, aq, bq, iq, k16n, fresh); break;
                        case 2: issue_stage<2>(tbuf, st_lo, aq, bq, iq, k16n, fresh); break;
                        case 3: issue_stage<3>(tbuf, st_lo, aq, bq, iq, k16n, fresh); break;
                        case 4: issue_stage<4>(tbuf, st_lo, aq, bq, iq, k16n, fresh); break;
                        case 5: issue_stage<5>(tbuf, st_lo, aq, bq, iq, k16n, fresh); break;
                        case 6: issue_stage<6>(tbuf, st_lo, aq, bq, iq, k16n, fresh); break;
                        case 7: issue_stage<7>(tbuf, st_lo, aq, bq, iq, k16n, fresh); break;
                        default: issue_stage<8>(tbuf, st_lo, aq, bq, iq, k16n, fresh); break;
                        }
                        mma_commit_elect(smem_u32(&empty_bar[s]));   // stage free once these MMAs finish
                    }
                }
                if (!ok) break;
                mma_commit_elect(smem_u32(&accf_bar[buf]));   // accumulator ready for the epilogue
                ++use[buf];
                nb = buf ^ 1;
            }
            if (!ok && lane == 0) s_wound = 1;
        }
    } else if (warp < EPI_WARPS) {
        // ---------------- epilogue: TMEM lane quarter q, column quarter h
        const int q = warp & 3, h = warp >> 2;
        int p = 0, nb = 0;
        uint32_t use[2] = {0u, 0u};
        int32_t n_act = 0;   // dose GEMM of a solver step: active (plan, point) pairs seen
        for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
            const Item w = decode_item<KIND>(s_start, s_per, s_nsplit, s_rows, kp.bn, p, item);
            p = w.p;
            const Prob &d = s_prob[p];
            const int n_rows = s_rows[p];
            const int buf = nb;
            const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BUF_COLS);
            bool ok = true;
            if constexpr (KIND == 1) {
                const int pt_i = w.sub * BM + q * 32 + lane;   // this thread's point (in the problem)
                const float4 pt = d.pt4[pt_i];                // D_min, D_max, scale, structure
                const int sv_own = (int)pt.w;
                // 32 points of one structure and bound pattern take that branch warp-uniformly
                const int c16 = (w.sub * BM + q * 32) / 16;
                const int i0 = d.chunk[c16], i1 = d.chunk[c16 + 1];
                const int mode = i0 == i1 ? (i0 & 7) : 0;
                const int sv = mode != 0 ? (i0 >> 3) : sv_own;
                asm volatile("bar.sync 1, %0;" ::"n"(EPI_WARPS * 32) : "memory");   // previous item's readers done
                if (threadIdx.x < BM) {   // all loads first (one round trip), then the stores
                    const int rr = threadIdx.x, rw = w.ptile * BM + rr;   // plan row of the tile
                    float c[8];
                    float4 sp[8];
#pragma unroll
                    for (int s2 = 0; s2 < 8; ++s2) {
                        const bool on = s2 < d.n_struct;
                        c[s2] = on && rw < n_rows ? d.Wc[(size_t)rw * d.n_struct + s2] : 0.0f;
                        sp[s2] = on ? d.sparams[s2] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    }
#pragma unroll
                    for (int s2 = 0; s2 < 8; ++s2) {
                        s_cl[s2][rr] = c[s2] * sp[s2].x;
                        s_ch[s2][rr] = c[s2] * sp[s2].w;
                    }
                }
                asm volatile("bar.sync 1, %0;" ::"n"(EPI_WARPS * 32) : "memory");
                // warp-uniform: tcgen05.ld below is warp-collective; every named barrier of this
                // loop is reached by all epilogue threads whatever the outcome
                ok = __all_sync(0xffffffffu,
                                mbar_wait(smem_u32(&accf_bar[buf]), use[buf] & 1u, kp.err, 3, kp.wait_ns));
                fence_after();
                if (ok) {
                    const bool has_dT = kp.has_dT != 0;
                    const bool wdose = kp.write_dose != 0;
                    const bool count = kp.sparse_ok && d.act != nullptr;
                    const bool sparse = s_sparse[p] != 0;
                    const float lo = pt.x, hi = pt.y, sc = pt.z;
                    const float *clr = s_cl[sv < 0 ? 0 : sv], *chr = s_ch[sv < 0 ? 0 : sv];
                    constexpr int CW = 8;                  // plan columns per TMEM load
#pragma unroll 1
                    for (int chk = 0; chk < BM / EPI_GROUPS / CW; ++chk) {
                        const int c = h * (BM / EPI_GROUPS) + chk * CW;   // first plan column
                        if (w.ptile * BM + c >= n_rows) break;   // no live plan left in this warp's columns
                        uint32_t dv[CW], ddv[CW];
#pragma unroll
                        for (int i = 0; i < CW; ++i) ddv[i] = 0u;
                        tmem_ld8(lane_addr + (uint32_t)c, dv);
                        if (has_dT) tmem_ld8(lane_addr + (uint32_t)(BM + c), ddv);
                        tmem_ld_wait_regs8(dv, ddv);
                        float out[CW], fv[CW], dfv[CW];
                        if ((mode == 1 || mode == 2) && !wdose) {
                            // one structure with one bound (warp-uniform): pairs of plan columns in
                            // packed FP32x2 arithmetic.  With s = +1 (lower bound) or -1 (upper):
                            // v = max(s (bound - d), 0), f = c v^2, dF/dd = -2 s c v, and the
                            // dose change's part f(d) - f(d - dd) = c dv (v + v_b), where dv is
                            // -s dd when both v, v_b > 0 and v - v_b otherwise (no cancellation)
                            const float sg = mode == 1 ? 1.0f : -1.0f;
                            const float bnd = mode == 1 ? lo : hi;
                            const float2 a2 = make_float2(-sg * sc, -sg * sc), b2 = make_float2(sg * bnd, sg * bnd);
                            const float2 s2 = make_float2(sg * sc, sg * sc), g2 = make_float2(-2.0f * sg * sc, -2.0f * sg * sc);
                            const float *wrow = mode == 1 ? clr : chr;
                            // a chunk whose 8 x 32 pairs all have v = v_b = 0 (most of them once
                            // the plans near their optima) gives zeros only: F and dF parts, dF/dd
                            bool act = false;
#pragma unroll
                            for (int i = 0; i < CW; i += 2) {
                                const float2 acc = make_float2(__uint_as_float(dv[i]), __uint_as_float(dv[i + 1]));
                                const float2 t = __ffma2_rn(a2, acc, b2);
                                act = act || t.x > 0.0f || t.y > 0.0f;
                                if (has_dT) {
                                    const float2 dacc = make_float2(__uint_as_float(ddv[i]), __uint_as_float(ddv[i + 1]));
                                    const float2 tb = __ffma2_rn(s2, dacc, t);
                                    act = act || tb.x > 0.0f || tb.y > 0.0f;
                                }
                            }
                            if (!__any_sync(0xffffffffu, act)) {
                                if ((lane & 3) == 0) {
                                    s_part[0][q][c + ((lane >> 2) & 7)] = 0.0f;
                                    s_part[1][q][c + ((lane >> 2) & 7)] = 0.0f;
                                }
                                const int row0 = w.ptile * BM + c;
                                if (count && sparse) {   // no active point: empty mask words
                                    if (lane < CW && row0 + lane < n_rows)
                                        d.mask[((size_t)(row0 + lane) * d.n_ptiles + w.sub) * 4 + q] = 0u;
                                    continue;
                                }
                                const int prow = lane >> 2, pseg = (lane & 3) * 8;   // as in the staged stores
                                if (row0 + prow < n_rows) {
                                    const size_t off = (size_t)(row0 + prow) * d.ld_g + w.sub * BM + q * 32 + pseg;
#pragma unroll
                                    for (int term = 0; term < 3; ++term)
                                        if (term < kp.nG)
                                            *reinterpret_cast<uint4 *>(d.G[term] + off) = make_uint4(0u, 0u, 0u, 0u);
                                }
                                continue;
                            }
#pragma unroll
                            for (int i = 0; i < CW; i += 2) {
                                const float2 acc = make_float2(__uint_as_float(dv[i]), __uint_as_float(dv[i + 1]));
                                const float2 cw = *reinterpret_cast<const float2 *>(wrow + c + i);
                                const float2 t = __ffma2_rn(a2, acc, b2);   // s (bound - d)
                                const float2 v = make_float2(fmaxf(t.x, 0.0f), fmaxf(t.y, 0.0f));
                                const float2 cv = __fmul2_rn(cw, v);
                                const float2 fq = __fmul2_rn(cv, v);
                                const float2 gq = __fmul2_rn(g2, cv);
                                fv[i] = fq.x;
                                fv[i + 1] = fq.y;
                                out[i] = gq.x;
                                out[i + 1] = gq.y;
                                dfv[i] = 0.0f;
                                dfv[i + 1] = 0.0f;
                                if (has_dT) {
                                    const float2 dacc = make_float2(__uint_as_float(ddv[i]), __uint_as_float(ddv[i + 1]));
                                    const float2 tb = __ffma2_rn(s2, dacc, t);   // s (bound - (d - dd))
                                    const float2 vb = make_float2(fmaxf(tb.x, 0.0f), fmaxf(tb.y, 0.0f));
                                    const float2 sdd = __fmul2_rn(s2, dacc);     // s dd
                                    const float2 dif = __fadd2_rn(v, make_float2(-vb.x, -vb.y));
                                    const float2 dl = make_float2((v.x > 0.0f && vb.x > 0.0f) ? -sdd.x : dif.x,
                                                                  (v.y > 0.0f && vb.y > 0.0f) ? -sdd.y : dif.y);
                                    const float2 dq = __fmul2_rn(__fmul2_rn(cw, dl), __fadd2_rn(v, vb));
                                    dfv[i] = dq.x;
                                    dfv[i + 1] = dq.y;
                                }
                            }
                        } else {
#pragma unroll
                        for (int i = 0; i < CW; ++i) {
                            const float dd0 = sc * __uint_as_float(dv[i]);
                            const float dd = sc * __uint_as_float(ddv[i]);
                            float f = 0.0f, df = 0.0f, gval = 0.0f;
                            if (mode == 1) {            // lower bound only
                                const float cl = clr[c + i];
                                const float u = fmaxf(lo - dd0, 0.0f);
                                f = cl * u * u;
                                gval = -2.0f * cl * u * sc;
                                if (has_dT) {
                                    // f(d) - f(d - dd) without cancellation (see eval_simt.cu)
                                    const float ub = fmaxf(lo - (dd0 - dd), 0.0f);
                                    const float dl = (u > 0.0f && ub > 0.0f) ? -dd : u - ub;
                                    df = cl * dl * (u + ub);
                                }
                            } else if (mode == 2) {     // upper bound only
                                const float ch = chr[c + i];
                                const float o = fmaxf(dd0 - hi, 0.0f);
                                f = ch * o * o;
                                gval = 2.0f * ch * o * sc;
                                if (has_dT) {
                                    const float ob = fmaxf((dd0 - dd) - hi, 0.0f);
                                    const float dh = (o > 0.0f && ob > 0.0f) ? dd : o - ob;
                                    df = ch * dh * (o + ob);
                                }
                            } else if (mode != 4 && sv >= 0) {   // both bounds, or mixed points
                                const float cl = clr[c + i], ch = chr[c + i];
                                const float u = fmaxf(lo - dd0, 0.0f), o = fmaxf(dd0 - hi, 0.0f);
                                f = cl * u * u + ch * o * o;
                                gval = 2.0f * (ch * o - cl * u) * sc;
                                if (has_dT) {
                                    const float db = dd0 - dd;
                                    const float ub = fmaxf(lo - db, 0.0f), ob = fmaxf(db - hi, 0.0f);
                                    const float dl = (u > 0.0f && ub > 0.0f) ? -dd : u - ub;
                                    const float dh = (o > 0.0f && ob > 0.0f) ? dd : o - ob;
                                    df = cl * dl * (u + ub) + ch * dh * (o + ob);
                                }
                            }
                            fv[i] = f;
                            dfv[i] = df;
                            out[i] = wdose ? dd0 : gval;
                        }
                        }
                        // per plan column: sum over this warp's 32 points, then over the lane
                        // quarters below (fixed order)
                        const float fsum = warp_col_sum8(fv, lane);
                        const float dfsum = has_dT ? warp_col_sum8(dfv, lane) : 0.0f;
                        if ((lane & 3) == 0) {
                            s_part[0][q][c + ((lane >> 2) & 7)] = fsum;
                            s_part[1][q][c + ((lane >> 2) & 7)] = dfsum;
                        }
                        // active pairs: dF/dd != 0 (a penalty term is on), live rows only
                        const int row0 = w.ptile * BM + c;
                        if (count && sparse) {
                            // this step's gradient is formed from the active pairs alone: per
                            // plan row, the mask word of these 32 points and their dF/dd in FP32
                            uint32_t mine = 0u;
#pragma unroll
                            for (int i = 0; i < CW; ++i) {
                                const uint32_t bal = __ballot_sync(0xffffffffu, out[i] != 0.0f);
                                if (lane == i) mine = bal;
                            }
                            if (lane < CW && row0 + lane < n_rows) {
                                d.mask[((size_t)(row0 + lane) * d.n_ptiles + w.sub) * 4 + q] = mine;
                                n_act += __popc(mine);
                            }
#pragma unroll
                            for (int i = 0; i < CW; ++i)
                                if (out[i] != 0.0f && row0 + i < n_rows)
                                    d.Gs[(size_t)(row0 + i) * d.ld_g + pt_i] = out[i];
                            continue;
                        }
                        if (count) {
#pragma unroll
                            for (int i = 0; i < CW; ++i) n_act += (out[i] != 0.0f && row0 + i < n_rows) ? 1 : 0;
                        }
                        if (wdose) {
                            // rows of the dose run over points: the 8 x 8 blocks of (plan, point)
                            // values are transposed within each group of 8 lanes, so that a lane
                            // writes 8 consecutive points of one plan
                            uint32_t wv[CW];
#pragma unroll
                            for (int i = 0; i < CW; ++i) wv[i] = __float_as_uint(out[i]);
                            transpose8(wv, lane);
                            const int row = w.ptile * BM + c + (lane & 7);
                            if (row < n_rows) {
                                const size_t off = (size_t)row * d.ld_g + w.sub * BM + q * 32 + (lane >> 3) * 8;
                                float4 *o4 = reinterpret_cast<float4 *>(d.dose_out + off);
                                o4[0] = make_float4(__uint_as_float(wv[0]), __uint_as_float(wv[1]),
                                                    __uint_as_float(wv[2]), __uint_as_float(wv[3]));
                                o4[1] = make_float4(__uint_as_float(wv[4]), __uint_as_float(wv[5]),
                                                    __uint_as_float(wv[6]), __uint_as_float(wv[7]));
                            }
                        } else {
                            // rows of G run over points: each BF16 term passes through this warp's
                            // 512 bytes of shared memory as [plan][point], from which every lane
                            // takes 8 consecutive points of one plan (one 16-byte store)
                            uint32_t t12[CW];   // terms 1 | 2, packed by one conversion
                            uint16_t t3[CW];    // term 3 (bf16x3)
#pragma unroll
                            for (int i = 0; i < CW; ++i) {
                                const float r1 = out[i] - __bfloat162float(__float2bfloat16_rn(out[i]));
                                const __nv_bfloat162 b12 = __floats2bfloat162_rn(out[i], r1);
                                t12[i] = *reinterpret_cast<const uint32_t *>(&b12);
                                t3[i] = kp.nG > 2 ? __bfloat16_as_ushort(__float2bfloat16_rn(r1 - __bfloat162float(b12.y)))
                                                  : (uint16_t)0;
                            }
                            uint16_t *stg = s_gst[warp];
                            const int prow = lane >> 2, pseg = (lane & 3) * 8;   // plan, first point written
                            const int row = w.ptile * BM + c + prow;
                            const size_t off = (size_t)row * d.ld_g + w.sub * BM + q * 32 + pseg;
#pragma unroll
                            for (int term = 0; term < 3; ++term) {
                                if (term >= kp.nG) break;
#pragma unroll
                                for (int i = 0; i < CW; ++i)
                                    stg[i * 32 + lane] = term == 0 ? (uint16_t)(t12[i] & 0xffffu)
                                                       : term == 1 ? (uint16_t)(t12[i] >> 16) : t3[i];
                                __syncwarp();
                                const uint4 v = *reinterpret_cast<const uint4 *>(stg + prow * 32 + pseg);
                                if (row < n_rows) *reinterpret_cast<uint4 *>(d.G[term] + off) = v;
                                __syncwarp();
                            }
                        }
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[buf])) : "memory");
                if (!ok && lane == 0) s_fail = 1;
                asm volatile("bar.sync 1, %0;" ::"n"(EPI_WARPS * 32) : "memory");
                ok = s_fail == 0;   // uniform over the epilogue warps (read after the barrier)
                if (threadIdx.x < BM && ok) {   // fixed-order sum of the four lane quarters
                    const int rr = threadIdx.x, row = w.ptile * BM + rr;
                    if (row < n_rows) {
                        d.Fpart[(size_t)row * d.n_ptiles + w.sub] =
                            ((s_part[0][0][rr] + s_part[0][1][rr]) + s_part[0][2][rr]) + s_part[0][3][rr];
                        if (kp.has_dT)
                            d.dFpart[(size_t)row * d.n_ptiles + w.sub] =
                                ((s_part[1][0][rr] + s_part[1][1][rr]) + s_part[1][2][rr]) + s_part[1][3][rr];
                    }
                }
            } else {
                const int dw = w.dt * BM + q * 32 + lane;   // this thread's dwell
                const bool dw_ok = dw < d.nd_pad;
                const int ncols = w.half ? 128 : kp.bn;
                const int cw = ncols / EPI_GROUPS;          // plan columns of this warp
                ok = __all_sync(0xffffffffu,
                                mbar_wait(smem_u32(&accf_bar[buf]), use[buf] & 1u, kp.err, 3, kp.wait_ns));
                fence_after();
                if (ok) {
                    float *out = d.gpart + (size_t)w.sub * n_rows * d.nd_pad + dw;
                    for (int c0 = h * cw; c0 < (h + 1) * cw; c0 += 16) {
                        uint32_t v[16];
                        tmem_ld16(lane_addr + (uint32_t)c0, v);
                        tmem_ld_wait();
                        const int row0 = w.ptile * kp.bn + c0;
#pragma unroll
                        for (int k = 0; k < 16; ++k)
                            if (dw_ok && row0 + k < n_rows) out[(size_t)(row0 + k) * d.nd_pad] = __uint_as_float(v[k]);
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[buf])) : "memory");
            }
            ++use[buf];
            nb = buf ^ 1;
            if (!ok) {
                if (lane == 0) s_wound = 1;
                break;
            }
        }
        if constexpr (KIND == 1) {
            if (kp.sparse_ok) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) n_act += __shfl_xor_sync(0xffffffffu, n_act, o);
                if (lane == 0 && n_act > 0) atomicAdd(&s_act, n_act);
            }
        }
    }
    fence_before();
    __syncthreads();
    if (s_wound) {
        // a wait gave up: before the CTA frees its TMEM and exits, wait (bounded) for the TMA
        // copies it armed and the MMAs it issued, which may still be writing its shared memory
        // and TMEM
        if (warp == W_TMA && lane == 0) {
            const int it = s_prod_it;
            for (int st = 0; st < kp.n_stages; ++st) {
                if (it <= st) continue;   // never armed
                const int last = it - 1 - ((it - 1 - st) % kp.n_stages);   // last arm of stage st
                mbar_wait(smem_u32(&full_bar[st]), (uint32_t)(last / kp.n_stages) & 1u, nullptr, 0,
                          kDrainNs);
            }
        } else if (warp == W_MMA) {
            // the commit's phase completes once every MMA issued before it has finished
            mma_commit_elect(smem_u32(&drain_bar));
            mbar_wait(smem_u32(&drain_bar), 0u, nullptr, 0, kDrainNs);
        }
        fence_before();
        __syncthreads();
    }
    if constexpr (KIND == 1) {
        // one count per CTA into the single problem's counter of this step
        if (threadIdx.x == 0 && kp.sparse_ok && s_prob[0].act && s_act > 0)
            atomicAdd(s_prob[0].act + kp.parity, s_act);
    }
    if (warp == W_TMEM) {
        fence_after();
        tmem_dealloc(tmem, (uint32_t)TMEM_COLS);
    }
}

// ------------------------------------------------------------------ operand preparation
// Row scale (power of two, so that A / s is exact) and the BF16 split terms of A / s; for the
// E4M3 form the single term is A / s rounded to E4M3 (stored as BF16, exactly).
__global__ void k_split_A(const float *__restrict__ A32, int64_t nd, int64_t nd_pad, int64_t kpad,
                          int32_t terms, int32_t fp8, float *__restrict__ scale,
                          __nv_bfloat16 *A1, __nv_bfloat16 *A2, __nv_bfloat16 *A3)
{
    const int64_t row = blockIdx.x;
    const float *a = A32 + row * nd_pad;
    __shared__ float red[128];
    float mx = 0.0f;
    for (int64_t l = threadIdx.x; l < nd; l += blockDim.x) mx = fmaxf(mx, a[l]);
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    mx = red[0];
    float s = 1.0f;
    if (mx > 0.0f) s = exp2f(ceilf(log2f(fp8 ? mx / 448.0f : mx)));
    if (threadIdx.x == 0) scale[row] = s;
    for (int64_t l = threadIdx.x; l < kpad; l += blockDim.x) {
        const float v = l < nd ? a[l] / s : 0.0f;   // exact: s is a power of two
        const size_t o = (size_t)row * kpad + l;
        if (fp8) {
            const __nv_fp8_e4m3 q(v);
            A1[o] = __float2bfloat16_rn(float(q));
            continue;
        }
        const __nv_bfloat16 t1 = __float2bfloat16_rn(v);
        A1[o] = t1;
        const float r1 = v - __bfloat162float(t1);
        if (terms > 1) {
            const __nv_bfloat16 t2 = __float2bfloat16_rn(r1);
            A2[o] = t2;
            if (terms > 2) A3[o] = __float2bfloat16_rn(r1 - __bfloat162float(t2));
        }
    }
}

// Per-point epilogue data of the dose GEMM: (D_min, D_max, scale, structure id).
__global__ void k_point_data(const int8_t *__restrict__ sid, const float4 *__restrict__ sparams,
                             const float *__restrict__ scale, int64_t np_pad, float4 *__restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np_pad) return;
    const int sv = sid[i];
    float4 v = make_float4(-INFINITY, INFINITY, 0.0f, 0.0f);
    if (sv >= 0) v = make_float4(sparams[sv].y, sparams[sv].z, scale[i], (float)sv);
    out[i] = v;
}

// Epilogue mode of each run of 16 points: 4 = nothing to score (padding, or a structure with
// both bounds infinite), 1 = one structure with a lower bound only, 2 = one structure with an
// upper bound only, 3 = one structure with both bounds, 0 = several structures.
__global__ void k_chunk_info(const int8_t *__restrict__ sid, const float4 *__restrict__ sparams,
                             int64_t n_chunks, int32_t *__restrict__ out)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n_chunks) return;
    const int s0 = sid[c * 16];
    bool same = true;
    for (int i = 1; i < 16; ++i) same = same && sid[c * 16 + i] == s0;
    int info = 0;
    if (same) {
        if (s0 < 0) {
            info = 4;
        } else {
            const bool lo = isfinite(sparams[s0].y), hi = isfinite(sparams[s0].z);
            const int mode = lo && hi ? 3 : lo ? 1 : hi ? 2 : 4;
            info = (s0 << 3) | mode;
        }
    }
    out[c] = info;
}

__global__ void k_transpose_bf16(const __nv_bfloat16 *__restrict__ in, int64_t rows, int64_t cols,
                                 __nv_bfloat16 *__restrict__ out)
{
    __shared__ __nv_bfloat16 tile[32][33];
    const int64_t c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, c = c0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < rows && c < cols) ? in[r * cols + c] : __float2bfloat16_rn(0.0f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[c * rows + r] = tile[threadIdx.x][k];
    }
}

// Trial point of each compact row, as in k_prep_fp32, written as BF16 split terms of t and
// two BF16 terms of dT.
__global__ void k_prep_tc(SolverState s, TcRows r, int32_t force_base)
{
    const int i = blockIdx.x;
    if (i >= *s.n_act) return;
    const int j = s.list[i];
    const bool trial = !force_base && s.state[j] == ST_TRIAL;
    const float a = trial ? (float)s.alpha[j] : 0.0f;
    const size_t pb = (size_t)j * s.nd_pad, cb = (size_t)i * r.ld;
    for (int64_t l = threadIdx.x; l < r.kpad; l += blockDim.x) {
        float t = 0.0f, dt = 0.0f;
        if (l < s.nd_pad) {
            const float xv = s.x[pb + l];
            float xt = xv;
            if (trial) {
                const float ap = a * s.p[pb + l];
                xt = xv + ap;
                dt = ap * (2.0f * xv + ap);
            }
            s.xt[pb + l] = xt;
            t = xt * xt;
        }
        const __nv_bfloat16 t1 = __float2bfloat16_rn(t);
        r.T[0][cb + l] = t1;
        const float r1 = t - __bfloat162float(t1);
        if (r.nT > 1) {
            const __nv_bfloat16 t2 = __float2bfloat16_rn(r1);
            r.T[1][cb + l] = t2;
            if (r.nT > 2) r.T[2][cb + l] = __float2bfloat16_rn(r1 - __bfloat162float(t2));
        }
        const __nv_bfloat16 d1 = __float2bfloat16_rn(dt);
        r.dT[0][cb + l] = d1;
        r.dT[1][cb + l] = __float2bfloat16_rn(dt - __bfloat162float(d1));
    }
    if (threadIdx.x < s.n_struct)
        r.Wc[(size_t)i * s.n_struct + threadIdx.x] = s.Wn[(size_t)j * s.n_struct + threadIdx.x];
    if (threadIdx.x == 0) s.slot_of[j] = i;
}

// ------------------------------------------------------------------ host helpers
// cuTensorMapEncodeTiled is resolved through the runtime's driver entry-point query, so the
// library does not link libcuda directly (it still needs the driver at run time).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

int n_t_terms(int tc_terms) { return std::max(tc_terms, 2); }

// pairs (i, j) of split terms kept in a product: i + j <= max(nA, nB) + 1 (1-based)
bool keep_pair(int i, int j, int nA, int nB) { return (i + 1) + (j + 1) <= std::max(nA, nB) + 1; }

KParams make_params(const TcLaunchSet &set, int kind, int parity, bool with_dT, bool write_dose,
                    bool zero_next)
{
    KParams k{};
    k.maps = kind == 1 ? set.maps1 : set.maps2;
    k.probs = kind == 1 ? static_cast<const void *>(set.dose) : static_cast<const void *>(set.grad);
    k.n_probs = set.n;
    k.parity = parity;
    k.has_dT = kind == 1 && with_dT ? 1 : 0;
    k.write_dose = write_dose ? 1 : 0;
    k.zero_next = zero_next ? 1 : 0;
    k.sparse_ok = zero_next ? 1 : 0;
    const int nA = set.tc_terms, nT = n_t_terms(nA);
    k.nG = nT;
    k.bn = kind == 1 ? BM : grad_bn(nA, set.grad_tile);
    // N-side slot j: dose GEMM T_j, with dT_j stacked behind it for the two terms of dT;
    // gradient GEMM G_j, both 128-row halves of a 256-plan tile
    auto slot_maps = [&](Group &g, int j) {
        const int b = g.n_b++;
        g.b_map[b][0] = 3 + j;
        g.b_roff[b][0] = 0;
        g.b_map[b][1] = -1;
        g.b_roff[b][1] = 0;
        if (kind == 1 && k.has_dT && j < 2) {
            g.b_map[b][1] = 6 + j;
        } else if (kind == 2 && k.bn == 256) {
            g.b_map[b][1] = 3 + j;
            g.b_roff[b][1] = 128;
        }
        return b;
    };
    auto slot_n = [&](int j) { return kind == 1 ? ((k.has_dT && j < 2) ? 256 : 128) : k.bn; };
    auto add_pair = [](Group &g, int a, int b, int n) {
        g.pair_a[g.n_pair] = a;
        g.pair_b[g.n_pair] = b;
        g.pair_n[g.n_pair++] = n;
    };
    const bool stacked = (kind == 1 && k.has_dT) || (kind == 2 && k.bn == 256);
    k.slot_bytes = stacked ? 2 * BOX : BOX;
    int npairs = 0;
    for (int i = 0; i < nA; ++i)
        for (int j = 0; j < nT; ++j) npairs += keep_pair(i, j, nA, nT);
    const bool merged = nA * BOX + nT * k.slot_bytes <= SMEM_BUDGET / 2 && npairs <= MAX_PAIRS;
    int max_a = 0, max_b = 0;
    if (merged) {
        // every term of a K block in one stage, each tile loaded once per K block; the
        // N = 256 products first (the first product starts the accumulator)
        k.n_groups = 1;
        Group &g = k.g[0];
        g = Group{};
        g.n_a = nA;
        for (int i = 0; i < nA; ++i) g.a_map[i] = i;
        for (int j = 0; j < nT; ++j) slot_maps(g, j);
        for (int wide = 1; wide >= 0; --wide)
            for (int j = 0; j < nT; ++j)
                for (int i = 0; i < nA; ++i)
                    if (keep_pair(i, j, nA, nT) && (slot_n(j) == 256) == (wide == 1))
                        add_pair(g, i, j, slot_n(j));
        max_a = nA;
        max_b = nT;
    } else {
        // one stage kind per N-side term j, with the M-side terms it pairs with
        k.n_groups = nT;
        for (int j = 0; j < nT; ++j) {
            Group &g = k.g[j];
            g = Group{};
            slot_maps(g, j);
            for (int i = 0; i < nA; ++i)
                if (keep_pair(i, j, nA, nT)) {
                    g.a_map[g.n_a] = i;
                    add_pair(g, g.n_a++, 0, slot_n(j));
                }
            max_a = std::max(max_a, g.n_a);
        }
        max_b = 1;
    }
    k.b_off = max_a * BOX;
    k.stage_bytes = k.b_off + max_b * k.slot_bytes;
    k.n_stages = std::max(1, std::min(MAX_STAGES, SMEM_BUDGET / k.stage_bytes));
    k.err = set.err;
    k.wait_ns = set.wait_ns;
    if (kind == 2)
        for (int r = 0; r < kTcPrefetch; ++r) {
            k.pf_ptr[r] = set.pf_ptr[r];
            k.pf_bytes[r] = set.pf_ptr[r] ? set.pf_bytes[r] & ~(int64_t)15 : 0;
        }
    return k;
}

size_t dyn_smem(const KParams &k) { return (size_t)k.n_stages * k.stage_bytes + 1024; }

cudaError_t ensure_attrs()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM_BUDGET + 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BUDGET + 1024);
    if (e != cudaSuccess) return e;
    done = true;
    return cudaSuccess;
}

int n16_of(const DevProblem &pb) { return (int)round_up(pb.n_dwell, 16); }

}  // namespace

// Plans per tile of the gradient GEMM: 128 when requested, else 256 when a merged stage of
// all terms fits twice in the ring (one MMA of N = 256 per product), else 128.
int grad_bn(int tc_terms, int requested)
{
    const int nA = tc_terms, nT = n_t_terms(tc_terms);
    const bool fits = (nA + 2 * nT) * BOX <= SMEM_BUDGET / 2;
    return requested == 128 || !fits ? 128 : 256;
}

bool tc_encode_map(CUtensorMap *m, const void *ptr, uint64_t cols, uint64_t rows,
                   uint32_t box_cols, uint32_t box_rows)
{
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t es[2] = {1, 1};
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
               es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int32_t tc_n_ptiles(const DevProblem &pb) { return (int32_t)(pb.np_pad / BM); }

int32_t tc_n_dtiles(const DevProblem &pb) { return (int32_t)ceil_div(pb.nd_pad, BM); }

double tc_mma_units(const DevProblem &pb, bool with_dT, int which)
{
    const int nA = pb.tc_terms, nT = n_t_terms(pb.tc_terms);
    int pairs = 0, with_dt_term = 0;
    for (int i = 0; i < nA; ++i)
        for (int j = 0; j < nT; ++j)
            if (keep_pair(i, j, nA, nT)) {
                ++pairs;
                with_dt_term += j < 2;   // these products also give A_i dT_j
            }
    return which == 1 ? pairs + (with_dT ? with_dt_term : 0) : pairs;
}
int32_t tc_max_split(const DevProblem &pb) { return (int32_t)std::min<int64_t>(148, pb.np_pad / BK); }

SplitPlan tc_split_plan(const DevProblem &pb, int32_t kb_per_split, int32_t grad_tile)
{
    SplitPlan p{};
    p.rows_per_tile = grad_bn(pb.tc_terms, grad_tile);
    p.other_tiles = tc_n_dtiles(pb);
    p.kb_total = (int32_t)(pb.np_pad / BK);
    if (kb_per_split > 0) {   // fixed split length: as many splits as that takes
        p.target_ctas = 1 << 30;
        p.max_split = (int32_t)ceil_div(p.kb_total, kb_per_split);
        p.min_kb = 1;
    } else {
        // about one wave of CTAs, but splits of at least 384 points: a few plan rows would
        // otherwise get up to 148 splits whose partial sums the step kernel adds (measured at
        // 1-256 plans of 12000 points: 384 points per split beat 128, 512 and longer ones)
        p.target_ctas = 148;
        p.max_split = tc_max_split(pb);
        p.min_kb = 6;
    }
    return p;
}

int64_t tc_launches_per_eval() { return 4; }

cudaError_t tc_prepare_problem(DevProblem *pb, int precision, cudaStream_t st,
                               const AllocFn &alloc)
{
    if (pb->n_dwell > 512 || pb->n_struct > 8) return cudaErrorNotSupported;
    const int terms = precision == GMCO_PREC_BF16X3 ? 3 : precision == GMCO_PREC_BF16X2 ? 2 : 1;
    pb->tc_terms = terms;
    pb->kpad = round_up(pb->n_dwell, BM);   // whole dwell tiles of the gradient GEMM
    const size_t n = (size_t)pb->np_pad * pb->kpad;
    for (int i = 0; i < terms; ++i) {
        cudaError_t e = alloc(reinterpret_cast<void **>(&pb->Ah[i]), n * sizeof(__nv_bfloat16));
        if (e != cudaSuccess) return e;
        e = alloc(reinterpret_cast<void **>(&pb->AhT[i]), n * sizeof(__nv_bfloat16));
        if (e != cudaSuccess) return e;
    }
    k_split_A<<<(unsigned)pb->np_pad, 128, 0, st>>>(pb->A32, pb->n_dwell, pb->nd_pad, pb->kpad,
                                                    terms, precision == GMCO_PREC_FP8 ? 1 : 0,
                                                    pb->row_scale, pb->Ah[0], pb->Ah[1], pb->Ah[2]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = alloc(reinterpret_cast<void **>(&pb->pt4), (size_t)pb->np_pad * sizeof(float4));
    if (e != cudaSuccess) return e;
    k_point_data<<<(unsigned)ceil_div(pb->np_pad, 256), 256, 0, st>>>(pb->sid, pb->sparams,
                                                                      pb->row_scale, pb->np_pad, pb->pt4);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = alloc(reinterpret_cast<void **>(&pb->chunk), (size_t)(pb->np_pad / 16) * sizeof(int32_t));
    if (e != cudaSuccess) return e;
    k_chunk_info<<<(unsigned)ceil_div(pb->np_pad / 16, 256), 256, 0, st>>>(pb->sid, pb->sparams,
                                                                          pb->np_pad / 16, pb->chunk);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int i = 0; i < terms; ++i) {
        dim3 grid((unsigned)ceil_div(pb->kpad, 32), (unsigned)ceil_div(pb->np_pad, 32));
        k_transpose_bf16<<<grid, dim3(32, 8), 0, st>>>(pb->Ah[i], pb->np_pad, pb->kpad, pb->AhT[i]);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return ensure_attrs();
}

TcDoseProb tc_dose_prob(const DevProblem &pb, const int32_t *cnt, const float *Wc,
                        __nv_bfloat16 *const *G, float *dose_out, float *Fpart, float *dFpart,
                        int32_t a_row, int32_t t_row, int32_t cap, int32_t ld_g)
{
    TcDoseProb d{};
    d.n_rows[0] = cnt;
    d.n_rows[1] = cnt + 1;
    d.pt4 = pb.pt4;
    d.chunk = pb.chunk;
    d.sparams = pb.sparams;
    d.Wc = Wc;
    for (int j = 0; j < 3; ++j) d.G[j] = j < n_t_terms(pb.tc_terms) ? G[j] : nullptr;
    d.dose_out = dose_out;
    d.Fpart = Fpart;
    d.dFpart = dFpart;
    d.a_row = a_row;
    d.t_row = t_row;
    d.kb = (int32_t)(pb.kpad / BK);
    d.k16 = n16_of(pb) / 16;
    d.n_ptiles = tc_n_ptiles(pb);
    d.n_struct = pb.n_struct;
    d.cap = cap;
    d.ld_g = ld_g;
    return d;
}

TcGradProb tc_grad_prob(const DevProblem &pb, const int32_t *cnt, float *gpart, SplitPlan sp,
                        int32_t at_row, int32_t g_row)
{
    TcGradProb d{};
    d.n_rows[0] = cnt;
    d.n_rows[1] = cnt + 1;
    d.gpart = gpart;
    d.sp = sp;
    d.at_row = at_row;
    d.g_row = g_row;
    d.kb = (int32_t)(pb.np_pad / BK);
    d.n_dt = tc_n_dtiles(pb);
    d.nd_pad = (int32_t)pb.nd_pad;
    return d;
}

cudaError_t tc_alloc(const DevProblem &pb, int32_t cap, float *Fpart, float *dFpart,
                     float *gpart, float *dose_out, const int32_t *cnt, int32_t split_kb,
                     int32_t grad_tile, int32_t sparse_permille, TcBuffers *b,
                     const AllocFn &alloc)
{
    *b = TcBuffers{};
    b->cap = cap;
    const int nT = n_t_terms(pb.tc_terms);
    const size_t tn = (size_t)cap * pb.kpad, gn = (size_t)cap * pb.np_pad;
    cudaError_t e;
    for (int j = 0; j < nT; ++j) {
        if ((e = alloc(reinterpret_cast<void **>(&b->T[j]), tn * 2)) != cudaSuccess) return e;
        if ((e = alloc(reinterpret_cast<void **>(&b->G[j]), gn * 2)) != cudaSuccess) return e;
    }
    for (int j = 0; j < 2; ++j) {
        if ((e = alloc(reinterpret_cast<void **>(&b->dT[j]), tn * 2)) != cudaSuccess) return e;
        if ((e = cudaMemset(b->dT[j], 0, tn * 2)) != cudaSuccess) return e;
    }
    if ((e = alloc(reinterpret_cast<void **>(&b->Wc), (size_t)cap * pb.n_struct * 4)) != cudaSuccess)
        return e;
    if ((e = alloc(reinterpret_cast<void **>(&b->err), 4)) != cudaSuccess) return e;
    if ((e = cudaMemset(b->err, 0, 4)) != cudaSuccess) return e;
    // operand maps
    bool ok = true;
    for (int i = 0; i < pb.tc_terms; ++i) {
        ok = ok && tc_encode_map(&b->maps1.m[i], pb.Ah[i], pb.kpad, pb.np_pad, kTcBoxCols, kTcBoxRowsA);
        ok = ok && tc_encode_map(&b->maps2.m[i], pb.AhT[i], pb.np_pad, pb.kpad, kTcBoxCols, kTcBoxRowsAT);
    }
    for (int j = 0; j < nT; ++j) {
        ok = ok && tc_encode_map(&b->maps1.m[3 + j], b->T[j], pb.kpad, cap, kTcBoxCols, kTcBoxRowsT);
        ok = ok && tc_encode_map(&b->maps2.m[3 + j], b->G[j], pb.np_pad, cap, kTcBoxCols, kTcBoxRowsG);
    }
    for (int j = 0; j < 2; ++j)
        ok = ok && tc_encode_map(&b->maps1.m[6 + j], b->dT[j], pb.kpad, cap, kTcBoxCols, kTcBoxRowsT);
    if (!ok) return cudaErrorInvalidValue;
    // descriptors of this problem alone
    b->Fpart = Fpart;
    b->dFpart = dFpart;
    b->gpart = gpart;
    b->dose_out = dose_out;
    b->cnt = cnt;
    b->sp = tc_split_plan(pb, split_kb, grad_tile);
    b->grad_tile = grad_bn(pb.tc_terms, grad_tile);
    TcDoseProb dp = tc_dose_prob(pb, cnt, b->Wc, b->G, dose_out, Fpart, dFpart, 0, 0, cap,
                                 (int32_t)pb.np_pad);
    TcGradProb gp = tc_grad_prob(pb, cnt, gpart, b->sp, 0, 0);
    if (sparse_permille > 0) {
        // active-set gradient: the FP32 dF/dd of the active pairs go to the dose buffer (a
        // solver step writes no dose); counts start with the first step on the dense path
        const size_t words = (size_t)cap * tc_n_ptiles(pb) * 4;
        if ((e = alloc(reinterpret_cast<void **>(&b->mask), words * 4)) != cudaSuccess) return e;
        if ((e = alloc(reinterpret_cast<void **>(&b->act), kTcActWords * 4)) != cudaSuccess) return e;
        if ((e = cudaMemset(b->mask, 0, words * 4)) != cudaSuccess) return e;
        if ((e = cudaMemset(b->act, 0, kTcActWords * 4)) != cudaSuccess) return e;
        b->Gs = dose_out;
        b->sp_thr = (int32_t)std::max<int64_t>(0, (int64_t)sparse_permille * pb.n_pnt / 1000);
        dp.mask = b->mask;
        dp.Gs = b->Gs;
        dp.act = b->act;
        dp.sp_thr = b->sp_thr;
        gp.act = b->act;
    }
    if ((e = alloc(reinterpret_cast<void **>(&b->d_dose), sizeof(TcDoseProb))) != cudaSuccess) return e;
    if ((e = alloc(reinterpret_cast<void **>(&b->d_grad), sizeof(TcGradProb))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b->d_dose, &dp, sizeof dp, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b->d_grad, &gp, sizeof gp, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    return cudaSuccess;
}

TcLaunchSet tc_single_set(const DevProblem &pb, const TcBuffers &b)
{
    TcLaunchSet set;
    set.maps1 = b.maps1;
    set.maps2 = b.maps2;
    set.dose = b.d_dose;
    set.grad = b.d_grad;
    set.n = 1;
    set.tc_terms = pb.tc_terms;
    set.err = b.err;
    set.wait_ns = b.wait_ns;
    set.max_items1 = ceil_div(b.cap, BM) * tc_n_ptiles(pb);
    set.grad_tile = b.grad_tile;
    set.max_items2 = ceil_div(b.cap, b.grad_tile) * tc_n_dtiles(pb) * b.sp.max_split;
    if (b.act) {
        set.gs_rows[0] = b.cnt;
        set.gs_rows[1] = b.cnt + 1;
        set.gs_mask = b.mask;
        set.gs_G = b.Gs;
        for (int j = 0; j < pb.tc_terms; ++j) set.gs_A[j] = pb.Ah[j];
        set.gs_act = b.act;
        set.gs_out = b.gpart;
        set.gs_ld = (int32_t)pb.np_pad;
        set.gs_nd = (int32_t)pb.nd_pad;
        set.gs_ptiles = tc_n_ptiles(pb);
        set.gs_kpad = (int32_t)pb.kpad;
        set.gs_terms = pb.tc_terms;
        set.gs_cap = b.cap;
    }
    return set;
}

TcRows tc_rows(const DevProblem &pb, const TcBuffers &b)
{
    TcRows r{};
    for (int j = 0; j < 3; ++j) r.T[j] = b.T[j];
    r.dT[0] = b.dT[0];
    r.dT[1] = b.dT[1];
    r.Wc = b.Wc;
    r.ld = (int32_t)pb.kpad;
    r.kpad = (int32_t)pb.kpad;
    r.nT = n_t_terms(pb.tc_terms);
    return r;
}

// ------------------------------------------------------------------ active-set gradient
// The A^T G part of the gradient, Eq. (2), from the active pairs only: g_j = sum over points i
// with dF/dd_i != 0 of dF/dd_i A_ij, the sum the gradient GEMM forms over every point, over the
// few points whose penalty term is on (their set shrinks to about 1% of a plan's points within a
// few tens of iterations).  One CTA of four warps per compact plan row.  In each pass every warp lists
// the active points of 2048 consecutive points from the dose epilogue's mask; the warps then
// share the pass's list (entry k to warp (k / BATCH) mod 4) and add the A rows of their
// entries; the four partial sums are added in warp order at the end.  CTA 0 also clears the
// next step's active-pair counter.
constexpr int kGsWarps = 4, kGsSeg = 2048, kGsPairs = 8;   // kpad <= 512

template <int NT>
__global__ void __launch_bounds__(kGsWarps * 32)
k_gsparse(const int32_t *__restrict__ rows, const uint32_t *__restrict__ mask,
          const float *__restrict__ G, const __nv_bfloat16 *__restrict__ A0,
          const __nv_bfloat16 *__restrict__ A1, const __nv_bfloat16 *__restrict__ A2,
          int32_t *act, float *__restrict__ out, int32_t ld, int32_t nd, int32_t n_ptiles,
          int32_t kpad, int32_t parity)
{
    constexpr int BATCH = NT == 3 ? 2 : 4;   // points in flight per warp
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        act[parity ^ 1] = 0;                 // next step's count
        if (act[2 + parity]) ++act[4];       // steps of this solve on this path
    }
    if (act[2 + parity] == 0) return;        // dense step (uniform over the grid)
    const int r = blockIdx.x;
    if (r >= *rows) return;                  // uniform over the CTA
    __shared__ int32_t s_pt[kGsWarps][kGsSeg];
    __shared__ int32_t s_n[kGsWarps];
    __shared__ float2 s_acc[kGsWarps - 1][kGsPairs][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint2 *mrow = reinterpret_cast<const uint2 *>(mask + (size_t)r * n_ptiles * 4);
    const int n2 = n_ptiles * 2;             // mask words of the row, in pairs
    const float *grow = G + (size_t)r * ld;
    const int kp = kpad / 64;                // dwell pairs per lane
    const __nv_bfloat16 *Aterm[3] = {A0, A1, A2};
    float2 acc[kGsPairs];
#pragma unroll
    for (int e = 0; e < kGsPairs; ++e) acc[e] = make_float2(0.0f, 0.0f);

    for (int pbase = 0; pbase < n2; pbase += kGsWarps * 32) {
        // this warp's 64 words (2048 points) of the pass: list its active points in order
        const int base = pbase + warp * 32;
        const uint2 wv = base + lane < n2 ? mrow[base + lane] : make_uint2(0u, 0u);
        const int c = __popc(wv.x) + __popc(wv.y);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int pos = incl - c;
        const int pt0 = (base + lane) * 64;   // first point of this lane's two words
        uint32_t w0 = wv.x, w1 = wv.y;
        while (w0) {
            s_pt[warp][pos++] = pt0 + __ffs(w0) - 1;
            w0 &= w0 - 1u;
        }
        while (w1) {
            s_pt[warp][pos++] = pt0 + 32 + __ffs(w1) - 1;
            w1 &= w1 - 1u;
        }
        if (lane == 31) s_n[warp] = incl;
        __syncthreads();
        const int c0 = s_n[0], c1 = c0 + s_n[1], c2 = c1 + s_n[2], E = c2 + s_n[3];
        for (int k0 = warp * BATCH; k0 < E; k0 += kGsWarps * BATCH) {
            int pj[BATCH];
            float gj[BATCH];
            __nv_bfloat162 v[BATCH][NT][kGsPairs];
#pragma unroll
            for (int j = 0; j < BATCH; ++j) {
                const int k = k0 + j < E ? k0 + j : k0;
                const int sg = k < c0 ? 0 : (k < c1 ? 1 : (k < c2 ? 2 : 3));
                const int off = k - (sg == 0 ? 0 : (sg == 1 ? c0 : (sg == 2 ? c1 : c2)));
                pj[j] = s_pt[sg][off];
            }
#pragma unroll
            for (int j = 0; j < BATCH; ++j) {
                gj[j] = k0 + j < E ? grow[pj[j]] : 0.0f;
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const __nv_bfloat162 *ar =
                        reinterpret_cast<const __nv_bfloat162 *>(Aterm[t] + (size_t)pj[j] * kpad) + lane;
#pragma unroll
                    for (int e = 0; e < kGsPairs; ++e)
                        if (e < kp) v[j][t][e] = ar[32 * e];
                }
            }
#pragma unroll
            for (int j = 0; j < BATCH; ++j)
#pragma unroll
                for (int e = 0; e < kGsPairs; ++e) {
                    if (e >= kp) continue;
                    float2 a = __bfloat1622float2(v[j][0][e]);
#pragma unroll
                    for (int t = 1; t < NT; ++t) {
                        const float2 b = __bfloat1622float2(v[j][t][e]);
                        a.x += b.x;
                        a.y += b.y;
                    }
                    acc[e].x = fmaf(gj[j], a.x, acc[e].x);
                    acc[e].y = fmaf(gj[j], a.y, acc[e].y);
                }
        }
        __syncthreads();   // the lists are rewritten by the next pass
    }
    if (warp > 0) {
#pragma unroll
        for (int e = 0; e < kGsPairs; ++e) s_acc[warp - 1][e][lane] = acc[e];
    }
    __syncthreads();
    if (warp == 0) {
        float *orow = out + (size_t)r * nd;
#pragma unroll
        for (int e = 0; e < kGsPairs; ++e) {
            const int dw = 64 * e + 2 * lane;
            if (e < kp && dw < nd) {
                float2 a = acc[e];
#pragma unroll
                for (int w = 0; w < kGsWarps - 1; ++w) {
                    a.x += s_acc[w][e][lane].x;
                    a.y += s_acc[w][e][lane].y;
                }
                *reinterpret_cast<float2 *>(orow + dw) = a;
            }
        }
    }
}

cudaError_t tc_launch_gemms(const TcLaunchSet &set, int32_t parity, bool with_dT,
                            bool write_dose, bool zero_next, cudaStream_t st,
                            int32_t *n_launches, cudaEvent_t *ev)
{
    int nl = 0;
    cudaError_t e = ensure_attrs();
    if (e != cudaSuccess) return e;
    if (set.n < 1 || set.n > kMaxMulti) return cudaErrorInvalidValue;
    const int n_sm = 148;
    const KParams k1 = make_params(set, 1, parity, with_dT, write_dose, zero_next);
    k_tc<1><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(n_sm, set.max_items1)), NTHREADS,
              dyn_smem(k1), st>>>(k1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ++nl;
    if (ev) cudaEventRecord(ev[2], st);
    if (!write_dose) {
        const KParams k2 = make_params(set, 2, parity, false, false, false);
        k_tc<2><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(n_sm, set.max_items2)), NTHREADS,
                  dyn_smem(k2), st>>>(k2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++nl;
        if (zero_next && set.gs_act) {   // solver step of a single problem with the active-set option
            const unsigned grid = (unsigned)set.gs_cap;   // one CTA per plan row
            const int32_t *rows = set.gs_rows[parity & 1];
            switch (set.gs_terms) {
            case 1:
                k_gsparse<1><<<grid, kGsWarps * 32, 0, st>>>(rows, set.gs_mask, set.gs_G, set.gs_A[0],
                                                          set.gs_A[0], set.gs_A[0], set.gs_act, set.gs_out,
                                                          set.gs_ld, set.gs_nd, set.gs_ptiles, set.gs_kpad, parity);
                break;
            case 2:
                k_gsparse<2><<<grid, kGsWarps * 32, 0, st>>>(rows, set.gs_mask, set.gs_G, set.gs_A[0],
                                                          set.gs_A[1], set.gs_A[1], set.gs_act, set.gs_out,
                                                          set.gs_ld, set.gs_nd, set.gs_ptiles, set.gs_kpad, parity);
                break;
            default:
                k_gsparse<3><<<grid, kGsWarps * 32, 0, st>>>(rows, set.gs_mask, set.gs_G, set.gs_A[0],
                                                          set.gs_A[1], set.gs_A[2], set.gs_act, set.gs_out,
                                                          set.gs_ld, set.gs_nd, set.gs_ptiles, set.gs_kpad, parity);
                break;
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            ++nl;
        }
    }
    *n_launches = nl;
    return cudaSuccess;
}

cudaError_t tc_launch_prep(const SolverState &s, const TcRows &r, int32_t cap, bool force_base,
                           cudaStream_t st)
{
    k_prep_tc<<<cap, 128, 0, st>>>(s, r, force_base ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t tc_launch_eval(const DevProblem &pb, const SolverState &s, const TcBuffers &b,
                           int32_t cap, bool with_dT, bool write_dose, bool force_base,
                           cudaStream_t st, int32_t *n_launches, cudaEvent_t *ev)
{
    int nl = 0;
    if (ev) cudaEventRecord(ev[0], st);
    cudaError_t e = tc_launch_prep(s, tc_rows(pb, b), cap, force_base, st);
    if (e != cudaSuccess) return e;
    ++nl;
    if (ev) cudaEventRecord(ev[1], st);
    int32_t ng = 0;
    if ((e = tc_launch_gemms(tc_single_set(pb, b), 0, with_dT, write_dose, false, st, &ng, ev)) !=
        cudaSuccess)
        return e;
    nl += ng;
    if (ev) cudaEventRecord(ev[3], st);
    EvalArgs fe{};
    fe.pb = pb;
    fe.n_rows = s.n_act;
    fe.cap = cap;
    fe.Fpart = b.Fpart;
    fe.dFpart = with_dT ? b.dFpart : nullptr;
    fe.gpart = write_dose ? nullptr : b.gpart;
    fe.sp = b.sp;
    if ((e = launch_finish(s, fe, tc_n_ptiles(pb), st)) != cudaSuccess) return e;
    ++nl;
    if (ev) cudaEventRecord(ev[4], st);
    *n_launches = nl;
    return cudaSuccess;
}

}  // namespace gmco
