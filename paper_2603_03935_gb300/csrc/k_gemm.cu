// D-weighted mask pooling as a tensor-core GEMM (Sec. III-C: each mask's
// embedding is the sum of its patches' features, each weighted by its
// distinctiveness D and its share of the mask).
//
//   E[m][d] = sum_p W[m][p] * F[p][d]      (W: pooling weights, F: tokens)
//
// computed as E^T = F^T W^T so the long token dimension D fills the 128 rows
// of one tcgen05 MMA and the masks (<= 256) form its N dimension:
//   A (128 x 32, K-major) = F^T tile  -- transposed while staged into shared memory
//   B (N   x 32, K-major) = W tile    -- W rows are already K-contiguous
// FP32 precision: the fp32 operands are split as x = hi + lo with hi, lo TF32
// and three kind::tf32 MMAs (hi*hi + hi*lo + lo*hi) accumulate in fp32 in
// TMEM, which keeps the fp32-level accuracy of the product (relative error
// ~1e-6).  BF16 precision: both operands rounded to bf16 (tokens given in
// bf16 are exact), one kind::f16 MMA per 16-wide K step, fp32 accumulation.
// FP8 precision: E4M3 operands with power-of-two scales, token p as
// rn(f_p / 2^a_p) and the weight rows prepared by the weights kernel, one
// kind::f8f6f4 MMA per 32-wide K step; the epilogue multiplies column m by
// its row scale 2^b_m.
//
// One CTA = one 128-row tile of D; one elected thread issues the MMAs; a
// two-stage shared-memory ring is recycled through mbarriers that
// tcgen05.commit arrives on.  Every wait is bounded by a global-timer limit
// after which the kernel records DISC_ERR_TIMEOUT and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "disc_common.cuh"
#include "kernels.h"

namespace disc {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Shared-memory matrix descriptor, SWIZZLE_NONE, K-major canonical layout:
// core matrices of 8 rows x 16 bytes stored contiguously (128 B); LBO = byte
// distance between core matrices adjacent along K, SBO = along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the tcgen05 family
    return d;                // base offset 0, absolute LBO mode, no swizzle
}

// Instruction descriptor of kind::tf32: D fp32, A/B tf32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Instruction descriptor of kind::f16 with bf16 A/B: D fp32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Instruction descriptor of kind::f8f6f4 with E4M3 A/B: D fp32, both K-major.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N)
{
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ uint32_t pack_e4m3(float a, float b, float c, float d)
{
    return (uint32_t)to_e4m3(a) | ((uint32_t)to_e4m3(b) << 8) | ((uint32_t)to_e4m3(c) << 16) |
           ((uint32_t)to_e4m3(d) << 24);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// bounded wait for the phase with the given parity; false after ~1 s
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    const uint64_t t0 = global_ns();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ float ldtok(const T* F, size_t i);
template <>
__device__ __forceinline__ float ldtok<float>(const float* F, size_t i) { return __ldg(F + i); }
template <>
__device__ __forceinline__ float ldtok<__nv_bfloat16>(const __nv_bfloat16* F, size_t i) { return __bfloat162float(F[i]); }

}  // namespace

constexpr uint32_t A_TILE_BYTES = GEMM_MT * GEMM_KC * 4;  // 16 KB (tf32); bf16 tiles take half, e4m3 a quarter
constexpr uint32_t A_LBO = (GEMM_MT / 8) * 128;           // 2048: next 16-byte K group (4 tf32 / 8 bf16 / 16 e4m3)

// two pipeline stages + barriers; the trailing guard keeps every address an
// MMA descriptor of this kernel can form inside the allocation
constexpr size_t GEMM_SMEM_GUARD = 48 * 1024;
constexpr size_t SMEM_MAX = 227 * 1024;
__host__ size_t gemm_smem_bytes(int NT)
{
    const size_t base = 2 * (2 * A_TILE_BYTES + 2 * (size_t)NT * GEMM_KC * 4) + 64;
    return std::min(base + GEMM_SMEM_GUARD, std::max(base, SMEM_MAX));
}

// Test hook: when set, the kernel issues no MMA and no commit, so its bounded
// waits run out and the frame fails with DISC_ERR_TIMEOUT (nothing is in
// flight when the tensor memory is freed).
__device__ int g_gemm_stall = 0;

cudaError_t set_gemm_stall(bool on)
{
    const int v = on ? 1 : 0;
    return cudaMemcpyToSymbol(g_gemm_stall, &v, sizeof(v));
}

// PR: the disc_precision of the frames this instance serves
template <typename T, int PR>
__global__ void __launch_bounds__(128, 1) k_pool_gemm(const FrameParams* fps, BatchScratch bs, int NT)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const FrameParams& fp = fps[blockIdx.y];
    const Scratch sc = bs.frame(blockIdx.y);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const T* F = (const T*)fp.tokens;
    const int D = fp.D, P = fp.P, M = fp.M;
    const int d0 = blockIdx.x * GEMM_MT;
    // uniform for the block: other dtype or precision, no masks, tile past D,
    // failed frame
    if (fp.token_bf16 != (sizeof(T) == 2) || fp.precision != PR || M <= 0 || d0 >= D || sc.ctr->err) return;

    // per stage: tf32 A hi | A lo | B hi | B lo, or bf16 / e4m3 A | B
    constexpr bool BF = PR == DISC_BF16, F8 = PR == DISC_FP8_E4M3;
    constexpr uint32_t EB = F8 ? 1 : (BF ? 2 : 4);  // operand bytes
    const uint32_t A_BYTES = A_TILE_BYTES / 4 * EB;
    const uint32_t B_TILE_BYTES = (uint32_t)NT * GEMM_KC * EB;
    const uint32_t B_LBO = (uint32_t)NT * 16;
    const uint32_t STAGE = (BF || F8) ? A_BYTES + B_TILE_BYTES : 2 * A_TILE_BYTES + 2 * B_TILE_BYTES;
    uint64_t* mbar = (uint64_t*)(smem + 2 * STAGE);
    uint32_t* tmem_slot = (uint32_t*)(mbar + 2);
    uint32_t ncols = 32;
    while (ncols < (uint32_t)NT) ncols <<= 1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = F8 ? idesc_e4m3(GEMM_MT, NT) : (BF ? idesc_bf16(GEMM_MT, NT) : idesc_tf32(GEMM_MT, NT));
    const int nchunks = (P + GEMM_KC - 1) / GEMM_KC;
    bool failed = false;
    int last_commit = -1;  // chunk of the most recent commit (same on all threads)
    const bool stall = g_gemm_stall != 0;  // uniform: read once
    // Thread tid stages row d0 + tid of the F^T tile: its 32 tokens of the
    // next chunk are loaded into registers while the current chunk is staged
    // and multiplied, so token loads stay in flight across the loop.
    auto load_chunk = [&](int c, float (&x)[GEMM_KC]) {
        const int d = d0 + tid, p0 = c * GEMM_KC;
#pragma unroll
        for (int j = 0; j < GEMM_KC; j++) {
            const int p = p0 + j;
            x[j] = (d < D && p < P) ? ldtok<T>(F, (size_t)p * D + d) : 0.0f;
        }
    };
    float xn[GEMM_KC];
    if (nchunks > 0) load_chunk(0, xn);

    for (int c = 0; c < nchunks && !failed; c++) {
        const int s = c & 1;
        uint8_t* st = smem + s * STAGE;
        float x[GEMM_KC];
#pragma unroll
        for (int j = 0; j < GEMM_KC; j++) x[j] = xn[j];
        if (c + 1 < nchunks) load_chunk(c + 1, xn);
        if (c >= 2) {
            // the MMAs of chunk c-2 read this stage: wait for their commit
            bool ok = mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((c >> 1) - 1) & 1));
            if (__syncthreads_or(!ok)) { failed = true; break; }
        }
        const int p0 = c * GEMM_KC;
        if constexpr (F8) {
            // A: F^T tile in e4m3, thread tid owns row d0 + tid, 16 patches per
            // 16 B; one exact multiply by 2^-a_p each
            {
                const float4* qm = (const float4*)(sc.qmul + p0);  // zero past P
#pragma unroll
                for (int q4 = 0; q4 < GEMM_KC / 4; q4++) {
                    const float4 mu = qm[q4];
                    x[4 * q4] = __fmul_rn(x[4 * q4], mu.x);
                    x[4 * q4 + 1] = __fmul_rn(x[4 * q4 + 1], mu.y);
                    x[4 * q4 + 2] = __fmul_rn(x[4 * q4 + 2], mu.z);
                    x[4 * q4 + 3] = __fmul_rn(x[4 * q4 + 3], mu.w);
                }
#pragma unroll
                for (int kq = 0; kq < GEMM_KC / 16; kq++) {
                    const float* y = x + 16 * kq;
                    const uint4 v = make_uint4(pack_e4m3(y[0], y[1], y[2], y[3]), pack_e4m3(y[4], y[5], y[6], y[7]),
                                               pack_e4m3(y[8], y[9], y[10], y[11]),
                                               pack_e4m3(y[12], y[13], y[14], y[15]));
                    *(uint4*)(st + kq * A_LBO + tid * 16) = v;
                }
            }
            // B: the e4m3 weight rows, NT rows x 32 patches
            {
                uint8_t* Bt = st + A_BYTES;
                for (int g = tid; g < NT * (GEMM_KC / 16); g += 128) {
                    const int n = g >> 1, kq = g & 1;
                    *(uint4*)(Bt + kq * B_LBO + n * 16) = *(const uint4*)(sc.W8 + (size_t)n * fp.Kpad + p0 + 16 * kq);
                }
            }
        } else if constexpr (BF) {
            // A: F^T tile in bf16, thread tid owns row d0 + tid, 8 patches per 16 B
            {
#pragma unroll
                for (int kq = 0; kq < GEMM_KC / 8; kq++) {
                    const float* y = x + 8 * kq;
                    const uint4 v = make_uint4(pack_bf16(y[0], y[1]), pack_bf16(y[2], y[3]), pack_bf16(y[4], y[5]),
                                               pack_bf16(y[6], y[7]));
                    *(uint4*)(st + kq * A_LBO + tid * 16) = v;
                }
            }
            // B: W tile in bf16, NT rows x 32 patches
            {
                uint8_t* Bt = st + A_BYTES;
                for (int g = tid; g < NT * (GEMM_KC / 8); g += 128) {
                    const int n = g >> 2, kq = g & 3;
                    const float4 x0 = *(const float4*)(sc.W + (size_t)n * fp.Kpad + p0 + 8 * kq);
                    const float4 x1 = *(const float4*)(sc.W + (size_t)n * fp.Kpad + p0 + 8 * kq + 4);
                    const uint4 v = make_uint4(pack_bf16(x0.x, x0.y), pack_bf16(x0.z, x0.w), pack_bf16(x1.x, x1.y),
                                               pack_bf16(x1.z, x1.w));
                    *(uint4*)(Bt + kq * B_LBO + n * 16) = v;
                }
            }
        } else {
        // A: F^T tile. Thread tid owns row r = tid (token dimension d0 + tid).
        {
            float* Ahi = (float*)st;
            float* Alo = (float*)(st + A_TILE_BYTES);
#pragma unroll
            for (int kq = 0; kq < GEMM_KC / 4; kq++) {
                const float* y = x + 4 * kq;
                float4 hi, lo;
                hi.x = tf32_rna(y[0]); lo.x = tf32_rna(y[0] - hi.x);
                hi.y = tf32_rna(y[1]); lo.y = tf32_rna(y[1] - hi.y);
                hi.z = tf32_rna(y[2]); lo.z = tf32_rna(y[2] - hi.z);
                hi.w = tf32_rna(y[3]); lo.w = tf32_rna(y[3] - hi.w);
                const uint32_t off = kq * A_LBO + tid * 16;
                *(float4*)((uint8_t*)Ahi + off) = hi;
                *(float4*)((uint8_t*)Alo + off) = lo;
            }
        }
        // B: W tile, NT rows x 32 patches, 16-byte granules
        {
            uint8_t* Bhi = st + 2 * A_TILE_BYTES;
            uint8_t* Blo = Bhi + B_TILE_BYTES;
            for (int g = tid; g < NT * (GEMM_KC / 4); g += 128) {
                const int n = g >> 3, kq = g & 7;
                float4 x = *(const float4*)(sc.W + (size_t)n * fp.Kpad + p0 + 4 * kq);
                float4 hi, lo;
                hi.x = tf32_rna(x.x); lo.x = tf32_rna(x.x - hi.x);
                hi.y = tf32_rna(x.y); lo.y = tf32_rna(x.y - hi.y);
                hi.z = tf32_rna(x.z); lo.z = tf32_rna(x.z - hi.z);
                hi.w = tf32_rna(x.w); lo.w = tf32_rna(x.w - hi.w);
                const uint32_t off = kq * B_LBO + n * 16;
                *(float4*)(Bhi + off) = hi;
                *(float4*)(Blo + off) = lo;
            }
        }
        }
        // make the generic-proxy stores visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && !stall) {
            fence_after();
            if constexpr (F8) {
                // one K step of 32 = two 16-byte core-matrix columns of e4m3
                const uint32_t a0 = smem_u32(st), b0 = a0 + A_BYTES;
                mma_e4m3(tmem, smem_desc(a0, A_LBO, 128), smem_desc(b0, B_LBO, 128), idesc, c > 0 ? 1u : 0u);
            } else if constexpr (BF) {
                // K step 16 = two 16-byte core-matrix columns of bf16
                const uint32_t a0 = smem_u32(st), b0 = a0 + A_BYTES;
#pragma unroll
                for (int ks = 0; ks < GEMM_KC / 16; ks++) {
                    const uint32_t ao = ks * 2 * A_LBO, bo = ks * 2 * B_LBO;
                    mma_bf16(tmem, smem_desc(a0 + ao, A_LBO, 128), smem_desc(b0 + bo, B_LBO, 128), idesc,
                             (c > 0 || ks > 0) ? 1u : 0u);
                }
            } else {
                const uint32_t a_hi = smem_u32(st), a_lo = a_hi + A_TILE_BYTES;
                const uint32_t b_hi = a_hi + 2 * A_TILE_BYTES, b_lo = b_hi + B_TILE_BYTES;
#pragma unroll
                for (int ks = 0; ks < GEMM_KC / 8; ks++) {
                    const uint32_t ao = ks * 2 * A_LBO, bo = ks * 2 * B_LBO;
                    const uint64_t dah = smem_desc(a_hi + ao, A_LBO, 128), dal = smem_desc(a_lo + ao, A_LBO, 128);
                    const uint64_t dbh = smem_desc(b_hi + bo, B_LBO, 128), dbl = smem_desc(b_lo + bo, B_LBO, 128);
                    mma_tf32(tmem, dah, dbh, idesc, (c > 0 || ks > 0) ? 1u : 0u);
                    mma_tf32(tmem, dah, dbl, idesc, 1u);
                    mma_tf32(tmem, dal, dbh, idesc, 1u);
                }
            }
            mma_commit(smem_u32(&mbar[s]));
        }
        if (!stall) last_commit = c;
    }
    if (!failed && nchunks > 0) {
        const int c = nchunks - 1;
        bool ok = mbar_wait(smem_u32(&mbar[c & 1]), (uint32_t)((c >> 1) & 1));
        failed = __syncthreads_or(!ok);
    }
    fence_after();
    if (!failed && nchunks > 0) {
        // epilogue: warp w reads TMEM lanes 32w..32w+31 (rows d0 + 32w + lane)
        const int d = d0 + warp * 32 + lane;
        for (int c0 = 0; c0 < NT; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int m = c0 + j;
                if (m < M && d < D) {
                    float v = __uint_as_float(r[j]);
                    if constexpr (F8) v = scale_pow2(v, sc.qexpm[m]);
                    sc.Efast[(size_t)m * D + d] = v;
                }
            }
        }
    } else if (failed) {
        // give MMAs still in flight one more bounded wait before TMEM is freed
        if (last_commit >= 0 && tid == 0)
            mbar_wait(smem_u32(&mbar[last_commit & 1]), (uint32_t)((last_commit >> 1) & 1));
        if (tid == 0) atomicCAS(&sc.ctr->err, 0, DISC_ERR_TIMEOUT);
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

int launch_pool_gemm(const FrameParams* fps, const BatchScratch& bs, int B, int D, int Mmax, const bool any[2][3],
                     cudaStream_t st)
{
    if (Mmax <= 0) return 0;
    const int NT = std::max(16, (Mmax + 15) / 16 * 16);
    const size_t smem = gemm_smem_bytes(NT);
    dim3 g((D + GEMM_MT - 1) / GEMM_MT, B);
    int n = 0;
    if (any[0][0]) { k_pool_gemm<float, DISC_FP32><<<g, 128, smem, st>>>(fps, bs, NT); n++; }
    if (any[1][0]) { k_pool_gemm<__nv_bfloat16, DISC_FP32><<<g, 128, smem, st>>>(fps, bs, NT); n++; }
    if (any[0][1]) { k_pool_gemm<float, DISC_BF16><<<g, 128, smem, st>>>(fps, bs, NT); n++; }
    if (any[1][1]) { k_pool_gemm<__nv_bfloat16, DISC_BF16><<<g, 128, smem, st>>>(fps, bs, NT); n++; }
    if (any[0][2]) { k_pool_gemm<float, DISC_FP8_E4M3><<<g, 128, smem, st>>>(fps, bs, NT); n++; }
    if (any[1][2]) { k_pool_gemm<__nv_bfloat16, DISC_FP8_E4M3><<<g, 128, smem, st>>>(fps, bs, NT); n++; }
    return n;
}

template <typename T, int PR>
static cudaError_t gemm_attr(int mx)
{
    return cudaFuncSetAttribute(k_pool_gemm<T, PR>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

cudaError_t set_gemm_kernel_attrs()
{
    const int mx = (int)gemm_smem_bytes(MAX_MASKS);
    cudaError_t e = gemm_attr<float, DISC_FP32>(mx);
    if (e == cudaSuccess) e = gemm_attr<__nv_bfloat16, DISC_FP32>(mx);
    if (e == cudaSuccess) e = gemm_attr<float, DISC_BF16>(mx);
    if (e == cudaSuccess) e = gemm_attr<__nv_bfloat16, DISC_BF16>(mx);
    if (e == cudaSuccess) e = gemm_attr<float, DISC_FP8_E4M3>(mx);
    if (e == cudaSuccess) e = gemm_attr<__nv_bfloat16, DISC_FP8_E4M3>(mx);
    return e;
}

}  // namespace disc
