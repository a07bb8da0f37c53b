// gmco_evaluate_noalloc: the FP32 objective and gradient evaluation for callers that must not
// allocate device memory while they run -- for example code that executes inside a
// preallocated memory budget, a real-time loop where cudaMalloc's implicit synchronisation is
// not acceptable, or an embedding application that owns every device allocation itself.
//
// It computes the same quantities as gmco_evaluate on an FP32-form problem (objective and
// dF/dx of every plan at given dwell weights) with the same dose and gradient kernels, but
// all of its scratch (squared dwell weights, per-point dF/dd, per-tile and per-split partial
// sums) lives in one file-scope device array of fixed size, so the call itself allocates
// nothing.  Inputs and outputs are the caller's device buffers.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace gmco {
namespace {

// Upper bound of the scratch one call may use.  Every GPU that loads the library holds this
// array until the process exits.
constexpr size_t kScratchBytes = 8u << 20;   // 8 MiB
constexpr int kMaxDevices = 64;
constexpr int32_t kSplit = 4;                 // point splits of the gradient GEMM

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host-side address of g_scratch on each device, resolved once per device.
void *g_addr[kMaxDevices] = {};
std::mutex g_mu;

size_t align256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

struct Layout {
    size_t n_rows, Tc, Wc, G, Fpart, gpart, total;
};

Layout layout(const DevProblem &pb, int64_t P, int32_t n_ptiles)
{
    Layout L{};
    size_t off = 0;
    L.n_rows = off; off += align256(sizeof(int32_t));
    L.Tc = off;     off += align256((size_t)P * pb.nd_pad * sizeof(float));
    L.Wc = off;     off += align256((size_t)P * pb.n_struct * sizeof(float));
    L.G = off;      off += align256((size_t)P * pb.np_pad * sizeof(float));
    L.Fpart = off;  off += align256((size_t)n_ptiles * P * sizeof(float));
    L.gpart = off;  off += align256((size_t)kSplit * P * pb.nd_pad * sizeof(float));
    L.total = off;
    return L;
}

// Row i of the scratch gets t = x^2 (padded dwells 0) and w / N_s; thread 0 of block 0 also
// writes the row count that the GEMM kernels read.
__global__ void k_na_prep(const float *__restrict__ X, const float *__restrict__ W,
                          const float *__restrict__ inv_count, int32_t P, int32_t nd,
                          int32_t nd_pad, int32_t S, float *__restrict__ Tc,
                          float *__restrict__ Wc, int32_t *n_rows)
{
    const int i = blockIdx.x;
    if (i == 0 && threadIdx.x == 0) *n_rows = P;
    for (int l = threadIdx.x; l < nd_pad; l += blockDim.x) {
        const float x = l < nd ? X[(size_t)i * nd + l] : 0.0f;
        Tc[(size_t)i * nd_pad + l] = x * x;
    }
    if (threadIdx.x < S) Wc[(size_t)i * S + threadIdx.x] = W[(size_t)i * S + threadIdx.x] * inv_count[threadIdx.x];
}

// F = fixed-order FP64 sum of the per-tile partials; dF/dx = 2 x * sum over the n_split
// splits that the gradient GEMM wrote (the same split plan decides both).
__global__ void k_na_finish(const float *__restrict__ X, const float *__restrict__ Fpart,
                            const float *__restrict__ gpart, int32_t P, int32_t nd,
                            int32_t nd_pad, int32_t n_ptiles, int32_t n_split,
                            double *__restrict__ F, float *__restrict__ grad)
{
    const int i = blockIdx.x;
    if (grad) {
        for (int l = threadIdx.x; l < nd; l += blockDim.x) {
            float acc = 0.0f;
            for (int q = 0; q < n_split; ++q) acc += gpart[((size_t)q * P + i) * nd_pad + l];
            grad[(size_t)i * nd + l] = 2.0f * X[(size_t)i * nd + l] * acc;
        }
    }
    if (threadIdx.x == 0 && F) {
        double f = 0.0;
        for (int t = 0; t < n_ptiles; ++t) f += (double)Fpart[(size_t)i * n_ptiles + t];
        F[i] = f;
    }
}

}  // namespace

// Resolves this device's address of g_scratch (once per device, with the device current).
cudaError_t noalloc_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

size_t noalloc_scratch_bytes() { return kScratchBytes; }

size_t noalloc_required_bytes(const DevProblem &pb, int64_t P)
{
    return layout(pb, P, simt_n_ptiles(pb)).total;
}

cudaError_t noalloc_evaluate(const DevProblem &pb, const float *W, int64_t P, const float *X,
                             double *F, float *grad, cudaStream_t st)
{
    void *base = nullptr;
    cudaError_t e = noalloc_scratch(&base);
    if (e != cudaSuccess) return e;
    const int32_t n_ptiles = simt_n_ptiles(pb);
    const Layout L = layout(pb, P, n_ptiles);
    if (L.total > kScratchBytes) return cudaErrorInvalidValue;
    unsigned char *b = static_cast<unsigned char *>(base);
    int32_t *n_rows = reinterpret_cast<int32_t *>(b + L.n_rows);
    float *Tc = reinterpret_cast<float *>(b + L.Tc);
    float *Wc = reinterpret_cast<float *>(b + L.Wc);
    EvalArgs ea{};
    ea.pb = pb;
    ea.n_rows = n_rows;
    ea.cap = (int32_t)P;
    ea.Tt = Tc;
    ea.dT = nullptr;
    ea.Wc = Wc;
    ea.G = reinterpret_cast<float *>(b + L.G);
    ea.Fpart = reinterpret_cast<float *>(b + L.Fpart);
    ea.dFpart = nullptr;
    ea.gpart = reinterpret_cast<float *>(b + L.gpart);
    ea.sp = simt_split_plan(pb);
    ea.sp.target_ctas = 1 << 30;     // at most kSplit point splits (the scratch holds that many)
    ea.sp.max_split = kSplit;
    ea.sp.min_kb = 1;
    // the splits the gradient GEMM writes: fewer than kSplit when the points fill fewer
    // K blocks; the finish kernel adds exactly these
    int32_t kbps = 0, n_split = 0;
    split_plan(ea.sp, (int32_t)P, &kbps, &n_split);
    if (n_split < 1 || n_split > kSplit) return cudaErrorInvalidValue;
    k_na_prep<<<(unsigned)P, 128, 0, st>>>(X, W, pb.inv_count, (int32_t)P, (int32_t)pb.n_dwell,
                                           (int32_t)pb.nd_pad, pb.n_struct, Tc, Wc, n_rows);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_gemm1_simt(ea, MODE_G, st)) != cudaSuccess) return e;
    if (grad && (e = launch_gemm2_simt(ea, st)) != cudaSuccess) return e;
    k_na_finish<<<(unsigned)P, 128, 0, st>>>(X, ea.Fpart, grad ? ea.gpart : nullptr, (int32_t)P,
                                             (int32_t)pb.n_dwell, (int32_t)pb.nd_pad, n_ptiles,
                                             n_split, F, grad);
    return cudaGetLastError();
}

}  // namespace gmco
