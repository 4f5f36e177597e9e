// Feature-side kernels of the integration step (Sec. III-C), batched over the
// frames of a batch (blockIdx.z = frame slot):
//   Eq. 1 distinctiveness map, mask->patch coverage, pooling weights with the
//   image-based quality terms (S_size, S_sem, S_dist of Eq. 2), and the exact
//   D-weighted pooled embedding.  None of them touches the map, so all frames
//   of a batch run in one launch.
#include <cuda_bf16.h>

#include "disc_common.cuh"
#include "kernels.h"

namespace disc {

template <typename T>
__device__ __forceinline__ float tok(const T* F, size_t i);
template <>
__device__ __forceinline__ float tok<float>(const float* F, size_t i) { return __ldg(F + i); }
template <>
__device__ __forceinline__ float tok<__nv_bfloat16>(const __nv_bfloat16* F, size_t i)
{
    return __bfloat162float(F[i]);
}

__device__ __forceinline__ void set_err(FrameCounters* c, int code) { atomicCAS(&c->err, 0, code); }

// ---- Eq. 1, pass 1: column sums of the tokens (mean token) + range check ----
template <typename T>
__global__ void k_tok_colsum(const FrameParams* fps, BatchScratch bs)
{
    const FrameParams& fp = fps[blockIdx.z];
    if (fp.token_bf16 != (sizeof(T) == 2)) return;
    const Scratch sc = bs.frame(blockIdx.z);
    const T* F = (const T*)fp.tokens;
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    const int p0 = blockIdx.y * 64, p1 = min(fp.P, p0 + 64);
    if (d >= fp.D || p0 >= fp.P) return;
    long long s = 0;
    bool bad = false;
    for (int p = p0; p < p1; p++) {
        float x = tok<T>(F, (size_t)p * fp.D + d);
        bad |= !(fabsf(x) <= TOKEN_LIMIT);
        s += fix32f(x, S_TOK);
    }
    atomicAdd((unsigned long long*)&sc.sumF[d], (unsigned long long)s);
    if (bad) set_err(sc.ctr, DISC_ERR_RANGE);
}

// ---- mean token, global embedding, ||g||^2 -----------------------------------
__global__ void k_tok_mean(const FrameParams* fps, BatchScratch bs)
{
    const FrameParams& fp = fps[blockIdx.z];
    const Scratch sc = bs.frame(blockIdx.z);
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    long long gg = 0;
    if (d < fp.D) {
        float fb = __double2float_rn(__ddiv_rn(unfix(sc.sumF[d], S_TOK), (double)fp.P));
        sc.fbar[d] = fb;
        float g = fb;
        if (fp.gembed) {
            g = fp.gembed[d];
            if (!(fabsf(g) <= TOKEN_LIMIT)) set_err(sc.ctr, DISC_ERR_RANGE);
        }
        sc.gvec[d] = g;
        gg = fix32f(__fmul_rn(g, g), S_SQ);
    }
    gg = warp_sum(gg);
    if ((threadIdx.x & 31) == 0 && gg) atomicAdd((unsigned long long*)sc.gg, (unsigned long long)gg);
}

// ---- Eq. 1, pass 2: residual norms, token . g, ||token||^2 (warp per patch) --
template <typename T>
__global__ void k_tok_rows(const FrameParams* fps, BatchScratch bs)
{
    const FrameParams& fp = fps[blockIdx.z];
    if (fp.token_bf16 != (sizeof(T) == 2)) return;
    const Scratch sc = bs.frame(blockIdx.z);
    const T* F = (const T*)fp.tokens;
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= fp.P || sc.ctr->err) return;
    long long ss = 0, dg = 0, ff = 0;
    float mx = 0.0f;
    for (int d = lane; d < fp.D; d += 32) {
        float f = tok<T>(F, (size_t)p * fp.D + d);
        float r = __fsub_rn(f, sc.fbar[d]);
        ss += fix32f(__fmul_rn(r, r), S_SQ);
        dg += fix32f(__fmul_rn(f, sc.gvec[d]), S_SQ);
        ff += fix32f(__fmul_rn(f, f), S_SQ);
        mx = fmaxf(mx, fabsf(f));
    }
    ss = warp_sum(ss);
    dg = warp_sum(dg);
    ff = warp_sum(ff);
    if (fp.precision == DISC_FP8_E4M3) {
        // the token's E4M3 operand q_p = rn(f_p / 2^e) and, from its actual
        // residue, bounds of ||2^e q_p - f_p|| and ||q_p||; fp32 sums of at
        // most D/32 + 5 levels stay within (1 + 2^-10) of the exact values
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        // (any e with max |f| <= 448 * 2^e serves; from -127 on, 2^-e is a
        // normal float, so the GEMM scales by one exact multiply)
        const int e = max(e4m3_exp(mx), -127);
        float se = 0.0f, sn = 0.0f;
        for (int d = lane; d < fp.D; d += 32) {
            const float f = tok<T>(F, (size_t)p * fp.D + d);
            const float q = from_e4m3(to_e4m3(scale_pow2(f, -e)));
            const float r = __fsub_rn(scale_pow2(q, e), f);
            se = __fadd_rn(se, __fmul_rn(r, r));
            sn = __fadd_rn(sn, __fmul_rn(q, q));
        }
        se = warp_sum(se);
        sn = warp_sum(sn);
        if (lane == 0) {
            sc.qexp[p] = e;
            sc.qmul[p] = __int_as_float((127 - e) << 23);
            sc.qerr[p] = __fmul_rn(sqrtf(se), 1.0f + 0x1p-10f);
            sc.qnrm[p] = __fmul_rn(sqrtf(sn), 1.0f + 0x1p-10f);
        }
    }
    if (lane == 0) {
        float n = __double2float_rn(__dsqrt_rn(unfix(ss, S_SQ)));
        sc.nrm[p] = n;
        sc.dotg[p] = dg;
        sc.ffp[p] = ff;
        sc.fnorm[p] = __double2float_rn(__dsqrt_rn(unfix(ff, S_SQ)));
        atomicAdd((unsigned long long*)sc.nsum, (unsigned long long)fix32f(n, S_NRM));
    }
}

// ---- Eq. 1, pass 3: D_p and cos(f_p, g) ----------------------------------------
__global__ void k_tok_finish(const FrameParams* fps, BatchScratch bs)
{
    const FrameParams& fp = fps[blockIdx.z];
    const Scratch sc = bs.frame(blockIdx.z);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= fp.P || sc.ctr->err) return;
    double nbar = __ddiv_rn(unfix(*sc.nsum, S_NRM), (double)fp.P);
    sc.Dp[p] = __double2float_rn(__ddiv_rn((double)sc.nrm[p], __dadd_rn(nbar, (double)fp.eps)));
    long long ff = sc.ffp[p], gg = *sc.gg;
    float c = 0.0f;
    if (ff != 0 && gg != 0)
        c = __double2float_rn(__ddiv_rn(unfix(sc.dotg[p], S_SQ),
                                        __dmul_rn(__dsqrt_rn(unfix(ff, S_SQ)), __dsqrt_rn(unfix(gg, S_SQ)))));
    sc.cosg[p] = c;
}

// ---- mask -> patch coverage: one block per patch row, shared histogram --------
// Rows v with floor(v * Ph / H) == i form the band of patch row i.
__global__ void k_coverage(const FrameParams* fps, BatchScratch bs)
{
    extern __shared__ int32_t hist[];  // [M][Pw]
    const FrameParams& fp = fps[blockIdx.z];
    const Scratch sc = bs.frame(blockIdx.z);
    const int i = blockIdx.x;
    const int M = fp.M, Pw = fp.Pw;
    if (M <= 0 || i >= fp.Ph) return;
    for (int j = threadIdx.x; j < M * Pw; j += blockDim.x) hist[j] = 0;
    __syncthreads();
    const int v0 = (i * fp.H + fp.Ph - 1) / fp.Ph;
    const int v1 = ((i + 1) * fp.H + fp.Ph - 1) / fp.Ph;
    const size_t b0 = (size_t)v0 * fp.W, b1 = (size_t)v1 * fp.W;
    for (size_t idx = b0 + threadIdx.x; idx < b1; idx += blockDim.x) {
        int lab = fp.labels[idx];
        if (lab >= 1 && lab <= M) {
            int u = (int)(idx % fp.W);
            atomicAdd(&hist[(lab - 1) * Pw + (u * Pw) / fp.W], 1);
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < M * Pw; j += blockDim.x) {
        int m = j / Pw, jj = j % Pw;
        sc.cov[(size_t)m * fp.P + i * Pw + jj] = hist[j];
    }
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        int s = 0;
        for (int jj = 0; jj < Pw; jj++) s += hist[m * Pw + jj];
        if (s) atomicAdd(&sc.npix[m], s);
    }
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    T s = 0;
    for (int i = 0; i < nw; i++) s += red[i];
    __syncthreads();
    return s;
}

__device__ __forceinline__ float block_max(float v, float* red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    float s = 0.0f;
    for (int i = 0; i < nw; i++) s = fmaxf(s, red[i]);
    __syncthreads();
    return s;
}

// FP8 precision: the weight row of mask m as E4M3 operands and the bound of
// the pooled embedding the tensor cores form from them.  Token p enters the
// GEMM as q_p = rn(f_p / 2^a_p), so its weight is scaled to w'_p = 2^a_p w_p
// (exact) and the row stored as r_p = rn(w'_p / 2^b); the GEMM returns
// 2^b sum_p r_p q_p.  Against e = sum_p w_p f_p its error is at most
//   sum_p |2^b r_p - w'_p| ||q_p||       (weight rounding)
// + sum_p w_p ||2^a_p q_p - f_p||         (token rounding)
// + g 2^b sum_p r_p ||q_p||               (accumulation)
// with g = (Kpad/32 + 2) 2^-12: an allowance of 12 bits per addition of a
// 32-deep MMA step into the accumulator, well below fp32's own rounding.
// The sum is taken in fp32 and widened by (1 + 2^-10).  Returns the bound.
__device__ float fp8_weights(const FrameParams& fp, const Scratch& sc, int m, const float* w, uint8_t* w8,
                             float* red)
{
    float mx = 0.0f;
    for (int p = threadIdx.x; p < fp.P; p += blockDim.x) mx = fmaxf(mx, scale_pow2(w[p], sc.qexp[p]));
    mx = block_max(mx, red);
    const int b = e4m3_exp(mx);
    float g1 = 0.0f, g2 = 0.0f, g3 = 0.0f;
    for (int p = threadIdx.x; p < fp.P; p += blockDim.x) {
        const float ws = scale_pow2(w[p], sc.qexp[p]);
        const uint8_t q = to_e4m3(scale_pow2(ws, -b));
        w8[p] = q;
        const float r = from_e4m3(q);
        g1 = __fadd_rn(g1, __fmul_rn(fabsf(__fsub_rn(scale_pow2(r, b), ws)), sc.qnrm[p]));
        g2 = __fadd_rn(g2, __fmul_rn(w[p], sc.qerr[p]));
        g3 = __fadd_rn(g3, __fmul_rn(r, sc.qnrm[p]));
    }
    g1 = block_sum(g1, red);
    g2 = block_sum(g2, red);
    g3 = block_sum(g3, red);
    if (threadIdx.x == 0) sc.qexpm[m] = b;
    const float gam = ldexpf((float)(fp.Kpad / 32 + 2), -12);
    return __fmul_rn(__fadd_rn(__fadd_rn(g1, g2), __fmul_rn(gam, scale_pow2(g3, b))), 1.0f + 0x1p-10f);
}

// ---- pooling weights and the image-based quality terms (one block per mask) ---
// a_p = c_p * D_p;  w_p = a_p / sum a  (sum a == 0, or the second grid's view:
// w_p = c_p / |M|);
// S_size = min(lambda |M| / (H W), 1);  S_dist = 0.5 + 0.5 * sum a / |M|;
// S_sem = clamp(sum c_p ReLU(cos(f_p, g)) / |M|, 0, 1).
__global__ void k_weights(const FrameParams* fps, BatchScratch bs)
{
    __shared__ long long red_ll[32];
    __shared__ float red_f[32];
    const FrameParams& fp = fps[blockIdx.z];
    const Scratch sc = bs.frame(blockIdx.z);
    const int m = blockIdx.x;
    if (m >= fp.M || sc.ctr->err) return;
    const int npix = sc.npix[m];
    float* w = sc.W + (size_t)m * fp.Kpad;
    float* S = sc.S + 5 * m;
    const int32_t* c = sc.cov + (size_t)m * fp.P;
    const bool fp8 = fp.precision == DISC_FP8_E4M3;
    uint8_t* w8 = sc.W8 + (size_t)m * fp.Kpad;
    if (npix < fp.min_px) {
        for (int p = threadIdx.x; p < fp.P; p += blockDim.x) {
            w[p] = 0.0f;
            if (fp8) w8[p] = 0;
        }
        if (threadIdx.x < 5) S[threadIdx.x] = 0.0f;
        if (threadIdx.x == 0) sc.Bm[m] = 0.0f;
        return;
    }
    long long A = 0, sem = 0;
    for (int p = threadIdx.x; p < fp.P; p += blockDim.x) {
        float cp = (float)c[p];
        A += fix32f(__fmul_rn(cp, sc.Dp[p]), S_A);
        float rc = sc.cosg[p] > 0.0f ? sc.cosg[p] : 0.0f;
        sem += fix32f(__fmul_rn(cp, rc), S_SEM);
    }
    A = block_sum(A, red_ll);
    sem = block_sum(sem, red_ll);
    const float Af = __double2float_rn(unfix(A, S_A));
    float bsum = 0.0f;
    for (int p = threadIdx.x; p < fp.P; p += blockDim.x) {
        float cp = (float)c[p];
        float wp = A > 0 && !fp.uniform_w ? __fdiv_rn(__fmul_rn(cp, sc.Dp[p]), Af) : __fdiv_rn(cp, (float)npix);
        w[p] = wp;
        bsum += wp * sc.fnorm[p];
    }
    bsum = block_sum(bsum, red_f);
    if (fp8) bsum = fp8_weights(fp, sc, m, w, w8, red_f);
    if (threadIdx.x == 0) {
        sc.Bm[m] = bsum;
        S[0] = fminf(__fdiv_rn(__fmul_rn(fp.lambda_size, (float)npix), (float)(fp.H * fp.W)), 1.0f);
        float Dbar = __double2float_rn(__ddiv_rn(unfix(A, S_A), (double)npix));
        S[3] = __fadd_rn(0.5f, __fmul_rn(0.5f, Dbar));
        float sm = __double2float_rn(__ddiv_rn(unfix(sem, S_SEM), (double)npix));
        S[2] = fminf(fmaxf(sm, 0.0f), 1.0f);
        S[1] = 0.0f;
        S[4] = 0.0f;
    }
}

// ---- exact D-weighted pooled embedding: e_m[d] = sum_p w_p f_p[d] -------------
// Each product is rounded to fp32 and added exactly in 2^-40 fixed point, so
// the patches can be visited in any order: the block first gathers the
// patches the mask covers, then every thread (one d) walks only those.
template <typename T>
__global__ void k_pool_exact(const FrameParams* fps, BatchScratch bs)
{
    extern __shared__ unsigned char pool_smem[];
    __shared__ int nnz;
    const FrameParams& fp = fps[blockIdx.z];
    if (fp.token_bf16 != (sizeof(T) == 2)) return;
    const Scratch sc = bs.frame(blockIdx.z);
    int* plist = (int*)pool_smem;                 // [P]
    float* wlist = (float*)(plist + fp.P);        // [P]
    const T* F = (const T*)fp.tokens;
    const int m = blockIdx.x;
    if (m >= fp.M || sc.ctr->err) return;
    const int d = blockIdx.y * blockDim.x + threadIdx.x;
    const bool ok = sc.npix[m] >= fp.min_px;
    if (threadIdx.x == 0) nnz = 0;
    __syncthreads();
    if (ok)
        for (int p = threadIdx.x; p < fp.P; p += blockDim.x) {
            float wp = sc.W[(size_t)m * fp.Kpad + p];
            if (wp != 0.0f) {
                int at = atomicAdd(&nnz, 1);
                plist[at] = p;
                wlist[at] = wp;
            }
        }
    __syncthreads();
    if (d >= fp.D) return;
    long long acc = 0;
    const int n = nnz;
    for (int i = 0; i < n; i++)
        acc += fix32f(__fmul_rn(wlist[i], tok<T>(F, (size_t)plist[i] * fp.D + d)), S_EMB);
    sc.Ecan[(size_t)m * fp.D + d] = __double2float_rn(unfix(acc, S_EMB));
}

// the sums the second grid's view accumulates per slot: column sums, pixel
// counts, ||g||^2 and the residual-norm sum (its counters are the primary's)
__global__ void k_view_clear(BatchScratch bs, int D, int MM)
{
    const Scratch sc = bs.frame(blockIdx.y);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(D, MM); i += gridDim.x * blockDim.x) {
        if (i < D) sc.sumF[i] = 0;
        if (i < MM) sc.npix[i] = 0;
        if (i == 0) {
            *sc.gg = 0;
            *sc.nsum = 0;
        }
    }
}

int launch_view_clear(const BatchScratch& bs, int B, int D, int MM, cudaStream_t st)
{
    k_view_clear<<<dim3(4, B), 256, 0, st>>>(bs, D, MM);
    return 1;
}

// ---- host launchers (each returns the number of kernels it enqueued) ----------
// Batched launchers cover B frame slots; P, D, Ph, Pw and Mmax bound the grids.
int launch_token_stats(const FrameParams* fps, const BatchScratch& bs, int B, int P, int D, bool any_bf16,
                       bool any_f32, cudaStream_t st)
{
    const dim3 b256(256);
    int n = 0;
    dim3 gcol((D + 255) / 256, (P + 63) / 64, B);
    if (any_f32) { k_tok_colsum<float><<<gcol, b256, 0, st>>>(fps, bs); n++; }
    if (any_bf16) { k_tok_colsum<__nv_bfloat16><<<gcol, b256, 0, st>>>(fps, bs); n++; }
    k_tok_mean<<<dim3((D + 255) / 256, 1, B), b256, 0, st>>>(fps, bs);
    n++;
    dim3 grow((P + 7) / 8, 1, B);
    if (any_f32) { k_tok_rows<float><<<grow, b256, 0, st>>>(fps, bs); n++; }
    if (any_bf16) { k_tok_rows<__nv_bfloat16><<<grow, b256, 0, st>>>(fps, bs); n++; }
    k_tok_finish<<<dim3((P + 255) / 256, 1, B), b256, 0, st>>>(fps, bs);
    return n + 1;
}

int launch_coverage(const FrameParams* fps, const BatchScratch& bs, int B, int Ph, int Pw, int Mmax, cudaStream_t st)
{
    if (Mmax <= 0) return 0;
    k_coverage<<<dim3(Ph, 1, B), 256, coverage_smem_bytes(Mmax, Pw), st>>>(fps, bs);
    return 1;
}

int launch_weights(const FrameParams* fps, const BatchScratch& bs, int B, int Mmax, cudaStream_t st)
{
    if (Mmax <= 0) return 0;
    k_weights<<<dim3(Mmax, 1, B), 256, 0, st>>>(fps, bs);
    return 1;
}

int launch_pool_exact(const FrameParams* fps, const BatchScratch& bs, int B, int P, int D, int Mmax, bool any_bf16,
                      bool any_f32, cudaStream_t st)
{
    if (Mmax <= 0) return 0;
    dim3 gp(Mmax, (D + 255) / 256, B);
    size_t psm = 8 * (size_t)P;
    int n = 0;
    if (any_f32) { k_pool_exact<float><<<gp, 256, psm, st>>>(fps, bs); n++; }
    if (any_bf16) { k_pool_exact<__nv_bfloat16><<<gp, 256, psm, st>>>(fps, bs); n++; }
    return n;
}

// the [M][Pw] coverage histogram of one block
size_t coverage_smem_bytes(int max_masks, int Pw) { return sizeof(int32_t) * (size_t)max_masks * Pw; }

cudaError_t set_feature_kernel_attrs(int max_dyn_smem)
{
    cudaError_t e = cudaFuncSetAttribute(k_coverage, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pool_exact<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pool_exact<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_dyn_smem);
    return e;
}

}  // namespace disc
