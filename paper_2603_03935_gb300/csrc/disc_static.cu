// Token statistics (distinctiveness map and cosine to the global embedding)
// for callers that cannot allocate device memory.
//
// Some callers run where cudaMalloc is not an option: code that must not
// change the device's memory footprint after start-up, allocator-less
// embedding layers, or hosts that hand the library only pre-registered
// buffers.  This entry point keeps its working set (the exact int64 sums and a
// few per-token vectors) in one file-scope __device__ array instead of
// allocating; the caller still passes the tokens and the two output arrays.
//
// The array is resident on every GPU that loads the library until the process
// exits, and all calls on one GPU share it, so calls whose GPU work overlaps
// (two streams, two host threads) race on it.  Its contents persist between
// calls; every call clears the sums it accumulates before using them.
#include <cstring>
#include <mutex>

#include "disc_common.cuh"
#include "kernels.h"

using namespace disc;

namespace {

constexpr int STATIC_MAX_D = 4096;
constexpr int STATIC_MAX_P = 16384;

// byte offsets inside the static array (all 256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_CTR = 0;                                              // FrameCounters
constexpr size_t OFF_GG = align256(OFF_CTR + sizeof(FrameCounters));       // long long
constexpr size_t OFF_NSUM = OFF_GG + 8;                                    // long long
constexpr size_t OFF_SUMF = align256(OFF_NSUM + 8);                        // long long [D]
constexpr size_t ZERO_BYTES = OFF_SUMF;                                    // + 8 * D
constexpr size_t OFF_FBAR = align256(OFF_SUMF + 8 * (size_t)STATIC_MAX_D); // float [D]
constexpr size_t OFF_GVEC = align256(OFF_FBAR + 4 * (size_t)STATIC_MAX_D); // float [D]
constexpr size_t OFF_DOTG = align256(OFF_GVEC + 4 * (size_t)STATIC_MAX_D); // long long [P]
constexpr size_t OFF_FFP = align256(OFF_DOTG + 8 * (size_t)STATIC_MAX_P);  // long long [P]
constexpr size_t OFF_NRM = align256(OFF_FFP + 8 * (size_t)STATIC_MAX_P);   // float [P]
constexpr size_t OFF_FNORM = align256(OFF_NRM + 4 * (size_t)STATIC_MAX_P); // float [P]
constexpr size_t OFF_COS = align256(OFF_FNORM + 4 * (size_t)STATIC_MAX_P);   // float [P] (heatmap)
constexpr size_t OFF_PARAMS = align256(OFF_COS + 4 * (size_t)STATIC_MAX_P);  // FrameParams
constexpr size_t STATIC_BYTES = align256(OFF_PARAMS + sizeof(FrameParams));

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_addr[MAX_DEVICES] = {};

}  // namespace

// The working set: ~450 KB, one copy per GPU that loads the library.
static __device__ __align__(256) unsigned char g_token_scratch[STATIC_BYTES];

// heat_p = D_p * cos(f_p, q), one fp32 rounding
__global__ void k_heat(float* heat, const float* cosq, int P)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) heat[p] = __fmul_rn(heat[p], cosq[p]);
}

// Eq. 1 and the token cosines on the static working set; cosg may point into
// the working set itself (offset OFF_COS, given as nullptr here)
static disc_status static_stats(const void* tokens, int32_t token_dtype, int32_t P, int32_t D,
                                const float* global_embed, float eps, float* Dp, float* cosg, void* cuda_stream,
                                unsigned char** base_out)
{
    if (!tokens || !Dp || P <= 0 || D <= 0) return DISC_ERR_INVALID_ARG;
    if (P > STATIC_MAX_P || D > STATIC_MAX_D) return DISC_ERR_INVALID_ARG;
    if (token_dtype != DISC_TOKENS_F32 && token_dtype != DISC_TOKENS_BF16) return DISC_ERR_INVALID_ARG;
    if (!(eps >= 0.0f)) return DISC_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return DISC_ERR_CUDA;
    }
    unsigned char* base = nullptr;
    {
        // once per device, with that device current: the device address of
        // the array (in host code its name is only a host-side stand-in)
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_token_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return DISC_ERR_CUDA;
            }
            g_addr[dev] = (unsigned char*)p;
        }
        base = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;

    FrameParams fp{};
    fp.P = P;
    fp.D = D;
    fp.eps = eps;
    fp.tokens = tokens;
    fp.token_bf16 = token_dtype == DISC_TOKENS_BF16;
    fp.gembed = global_embed;
    BatchScratch bs{};  // one frame slot: every stride stays zero
    Scratch& sc = bs.base;
    sc.ctr = (FrameCounters*)(base + OFF_CTR);
    sc.gg = (long long*)(base + OFF_GG);
    sc.nsum = (long long*)(base + OFF_NSUM);
    sc.sumF = (long long*)(base + OFF_SUMF);
    sc.fbar = (float*)(base + OFF_FBAR);
    sc.gvec = (float*)(base + OFF_GVEC);
    sc.dotg = (long long*)(base + OFF_DOTG);
    sc.ffp = (long long*)(base + OFF_FFP);
    sc.nrm = (float*)(base + OFF_NRM);
    sc.fnorm = (float*)(base + OFF_FNORM);
    sc.Dp = Dp;
    sc.cosg = cosg ? cosg : (float*)(base + OFF_COS);
    *base_out = base;

    // counters, ||g||^2, the residual-norm sum and the column sums start at
    // zero; the frame parameters travel to the array as well (pageable
    // source: staged before the call returns)
    FrameParams* dfp = (FrameParams*)(base + OFF_PARAMS);
    if (cudaMemsetAsync(base, 0, ZERO_BYTES + 8 * (size_t)D, st) != cudaSuccess ||
        cudaMemcpyAsync(dfp, &fp, sizeof(fp), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return DISC_ERR_CUDA;
    }
    const bool bf16 = token_dtype == DISC_TOKENS_BF16;
    launch_token_stats(dfp, bs, 1, P, D, bf16, !bf16, st);
    if (cudaGetLastError() != cudaSuccess) return DISC_ERR_CUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, &sc.ctr->err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return DISC_ERR_CUDA;
    }
    return (disc_status)err;
}

extern "C" disc_status disc_token_stats_static(const void* tokens, int32_t token_dtype, int32_t P, int32_t D,
                                               const float* global_embed, float eps, float* Dp, float* cosg,
                                               void* cuda_stream)
{
    if (!cosg) return DISC_ERR_INVALID_ARG;
    unsigned char* base = nullptr;
    return static_stats(tokens, token_dtype, P, D, global_embed, eps, Dp, cosg, cuda_stream, &base);
}

// Fig. 2: Eq. 1 with the query in the place of the global embedding gives D_p
// (written straight into heat) and cos(f_p, q); the heatmap is their product.
extern "C" disc_status disc_query_heatmap(const void* tokens, int32_t token_dtype, int32_t P, int32_t D,
                                          const float* query, float eps, float* heat, void* cuda_stream)
{
    if (!query || !heat) return DISC_ERR_INVALID_ARG;
    unsigned char* base = nullptr;
    disc_status s = static_stats(tokens, token_dtype, P, D, query, eps, heat, nullptr, cuda_stream, &base);
    if (s != DISC_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    k_heat<<<(P + 255) / 256, 256, 0, st>>>(heat, (const float*)(base + OFF_COS), P);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return DISC_ERR_CUDA;
    }
    return DISC_OK;
}
