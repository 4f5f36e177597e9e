// Feature-side kernels of the integration step (Sec. III-C):
//   Eq. 1 distinctiveness map, mask->patch coverage, pooling weights with the
//   image-based quality terms (S_size, S_sem, S_dist of Eq. 2), and the exact
//   D-weighted pooled embedding.
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
__global__ void k_tok_colsum(FrameParams fp, Scratch sc)
{
    const T* F = (const T*)fp.tokens;
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    const int p0 = blockIdx.y * 64, p1 = min(fp.P, p0 + 64);
    if (d >= fp.D) return;
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
__global__ void k_tok_mean(FrameParams fp, Scratch sc)
{
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
__global__ void k_tok_rows(FrameParams fp, Scratch sc)
{
    const T* F = (const T*)fp.tokens;
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= fp.P || sc.ctr->err) return;
    long long ss = 0, dg = 0, ff = 0;
    for (int d = lane; d < fp.D; d += 32) {
        float f = tok<T>(F, (size_t)p * fp.D + d);
        float r = __fsub_rn(f, sc.fbar[d]);
        ss += fix32f(__fmul_rn(r, r), S_SQ);
        dg += fix32f(__fmul_rn(f, sc.gvec[d]), S_SQ);
        ff += fix32f(__fmul_rn(f, f), S_SQ);
    }
    ss = warp_sum(ss);
    dg = warp_sum(dg);
    ff = warp_sum(ff);
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
__global__ void k_tok_finish(FrameParams fp, Scratch sc)
{
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
__global__ void k_coverage(FrameParams fp, Scratch sc)
{
    extern __shared__ int32_t hist[];  // [M][Pw]
    const int i = blockIdx.x;
    const int M = fp.M, Pw = fp.Pw;
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

// Fallback when [M][Pw] does not fit in shared memory: global atomics.
__global__ void k_coverage_global(FrameParams fp, Scratch sc)
{
    const size_t n = (size_t)fp.H * fp.W;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        int lab = fp.labels[idx];
        if (lab >= 1 && lab <= fp.M) {
            int v = (int)(idx / fp.W), u = (int)(idx % fp.W);
            int p = ((v * fp.Ph) / fp.H) * fp.Pw + (u * fp.Pw) / fp.W;
            atomicAdd(&sc.cov[(size_t)(lab - 1) * fp.P + p], 1);
            atomicAdd(&sc.npix[lab - 1], 1);
        }
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

// ---- pooling weights and the image-based quality terms (one block per mask) ---
// a_p = c_p * D_p;  w_p = a_p / sum a  (sum a == 0: w_p = c_p / |M|);
// S_size = min(lambda |M| / (H W), 1);  S_dist = 0.5 + 0.5 * sum a / |M|;
// S_sem = clamp(sum c_p ReLU(cos(f_p, g)) / |M|, 0, 1).
__global__ void k_weights(FrameParams fp, Scratch sc)
{
    __shared__ long long red_ll[32];
    __shared__ float red_f[32];
    const int m = blockIdx.x;
    if (sc.ctr->err) return;
    const int npix = sc.npix[m];
    float* w = sc.W + (size_t)m * fp.Kpad;
    float* S = sc.S + 5 * m;
    const int32_t* c = sc.cov + (size_t)m * fp.P;
    if (npix < fp.min_px) {
        for (int p = threadIdx.x; p < fp.P; p += blockDim.x) w[p] = 0.0f;
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
        float wp = A > 0 ? __fdiv_rn(__fmul_rn(cp, sc.Dp[p]), Af) : __fdiv_rn(cp, (float)npix);
        w[p] = wp;
        bsum += wp * sc.fnorm[p];
    }
    bsum = block_sum(bsum, red_f);
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
// Each product is rounded to fp32 and added exactly in 2^-40 fixed point.
template <typename T>
__global__ void k_pool_exact(FrameParams fp, Scratch sc)
{
    extern __shared__ float wrow[];  // [P]
    const T* F = (const T*)fp.tokens;
    const int m = blockIdx.x;
    const int d = blockIdx.y * blockDim.x + threadIdx.x;
    if (sc.ctr->err) return;
    const bool ok = sc.npix[m] >= fp.min_px;
    for (int p = threadIdx.x; p < fp.P; p += blockDim.x) wrow[p] = ok ? sc.W[(size_t)m * fp.Kpad + p] : 0.0f;
    __syncthreads();
    if (d >= fp.D) return;
    long long acc = 0;
    if (ok)
        for (int p = 0; p < fp.P; p++) {
            float wp = wrow[p];
            if (wp != 0.0f) acc += fix32f(__fmul_rn(wp, tok<T>(F, (size_t)p * fp.D + d)), S_EMB);
        }
    sc.Ecan[(size_t)m * fp.D + d] = __double2float_rn(unfix(acc, S_EMB));
}

// ---- host launchers (each returns the number of kernels it enqueued) ----------
int launch_token_stats(const FrameParams& fp, const Scratch& sc, cudaStream_t st)
{
    const dim3 b256(256);
    dim3 gcol((fp.D + 255) / 256, (fp.P + 63) / 64);
    if (fp.token_bf16) k_tok_colsum<__nv_bfloat16><<<gcol, b256, 0, st>>>(fp, sc);
    else k_tok_colsum<float><<<gcol, b256, 0, st>>>(fp, sc);
    k_tok_mean<<<(fp.D + 255) / 256, b256, 0, st>>>(fp, sc);
    if (fp.token_bf16) k_tok_rows<__nv_bfloat16><<<(fp.P + 7) / 8, b256, 0, st>>>(fp, sc);
    else k_tok_rows<float><<<(fp.P + 7) / 8, b256, 0, st>>>(fp, sc);
    k_tok_finish<<<(fp.P + 255) / 256, b256, 0, st>>>(fp, sc);
    return 4;
}

int launch_coverage(const FrameParams& fp, const Scratch& sc, cudaStream_t st, int cov_smem_limit)
{
    if (fp.M <= 0) return 0;
    size_t hsm = sizeof(int32_t) * (size_t)fp.M * fp.Pw;
    if ((int)hsm <= cov_smem_limit) {
        k_coverage<<<fp.Ph, 256, hsm, st>>>(fp, sc);
    } else {
        cudaMemsetAsync(sc.cov, 0, sizeof(int32_t) * (size_t)fp.M * fp.P, st);
        k_coverage_global<<<608, 256, 0, st>>>(fp, sc);
    }
    return 1;
}

int launch_weights(const FrameParams& fp, const Scratch& sc, cudaStream_t st)
{
    if (fp.M <= 0) return 0;
    k_weights<<<fp.M, 256, 0, st>>>(fp, sc);
    return 1;
}

int launch_pool_exact(const FrameParams& fp, const Scratch& sc, cudaStream_t st)
{
    if (fp.M <= 0) return 0;
    dim3 gp(fp.M, (fp.D + 255) / 256);
    size_t psm = sizeof(float) * (size_t)fp.P;
    if (fp.token_bf16) k_pool_exact<__nv_bfloat16><<<gp, 256, psm, st>>>(fp, sc);
    else k_pool_exact<float><<<gp, 256, psm, st>>>(fp, sc);
    return 1;
}

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
