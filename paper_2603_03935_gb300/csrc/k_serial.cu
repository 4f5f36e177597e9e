// The stateful part of the integration step, run frame after frame in order
// (each frame sees the map its predecessors left).  Per frame, four kernels
// (captured with the rest of the batch in one CUDA graph):
//   k_overlap  Sec. III-B  exact overlap histogram ov[m][k] of every segment
//                          with the instances of the map before this frame
//   k_score    Sec. III-B  geometry gate (overlap coefficient) and cosine gate
//                          per (segment, instance) pair; fast tensor-core
//                          score, exact re-score inside its error band
//   k_union    Sec. III-B  union of segments and instances (representative =
//              Sec. III-C  smallest id), new ids, merges, Q-replacement fusion
//                          (one CTA)
//   k_apply    Sec. III-B  embedding copies, insertion of the new voxels,
//                          flattening of the parent table, cleanup
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>

#include "disc_common.cuh"
#include "kernels.h"

namespace disc {

__device__ __forceinline__ void set_err(FrameCounters* c, int code) { atomicCAS(&c->err, 0, code); }

// ---- overlap histogram -----------------------------------------------------------
// Each block takes 1024 entries at a time.  Their (segment, root) pairs are
// counted in a shared-memory hash first; only the block's distinct pairs
// then update the frame's global histogram.  Voxels absent from the map go
// to the new-voxel hash with the lowest segment that contains them.
constexpr int SER_THREADS = 1024;
constexpr int OV_SLOTS = 2 * SER_THREADS;

// label of a key in the voxel table, -1 if absent
__device__ __forceinline__ int vt_label(const VoxelTable& vt, unsigned long long key)
{
    unsigned long long h = mix64(key) & vt.mask;
    for (unsigned long long pr = 0; pr <= vt.mask; pr++) {
        const unsigned long long kk = vt.keys[h];
        if (kk == key) return vt.labels[h];
        if (kk == EMPTY_KEY) return -1;
        h = (h + 1) & vt.mask;
    }
    return -1;
}

// cnt more voxels of segment-instance pair okey in the frame's pair hash
__device__ void add_pair(const Scratch& sc, const SerialScratch& ss, unsigned long long okey, int cnt = 1)
{
    unsigned long long t = mix64(okey) & ss.omask;
    for (unsigned long long pr = 0;; pr++) {
        const unsigned long long cur = ss.okeys[t];
        if (cur == okey) break;
        if (cur == EMPTY_KEY) {
            const unsigned long long prev = atomicCAS(&ss.okeys[t], EMPTY_KEY, okey);
            if (prev == EMPTY_KEY) {
                ss.olist[atomicAdd(&sc.ctr->n_pairs, 1)] = (int)t;
                break;
            }
            if (prev == okey) break;
        }
        t = (t + 1) & ss.omask;
        if (pr > ss.omask) {
            set_err(sc.ctr, DISC_ERR_TABLE_FULL);
            return;
        }
    }
    atomicAdd(&ss.ocnt[t], cnt);
}

// Neighbourhood overlap (overlap_dilation): segment voxel `key` (label lab,
// -1 if absent) overlaps each distinct instance labelling it or one of its 26
// neighbours, once.  One entry may add up to 27 pairs, so they go straight to
// the frame's pair hash.
__device__ void dilated_pairs(const Scratch& sc, const SerialScratch& ss, const VoxelTable& vt, const Instances& inst,
                              int m, unsigned long long key, int lab)
{
    int roots[27];
    int nr = 0;
    if (lab >= 0) roots[nr++] = inst.parent[lab];
    int k[3];
    unpack_key(key, k);
    // nine neighbours at a time (one x offset): every first probe slot loaded
    // at once; only a collision walks on
    for (int dx = -1; dx <= 1; dx++) {
        unsigned long long nk[9], cur[9];
        unsigned long long h[9];
        bool in[9];
#pragma unroll
        for (int j = 0; j < 9; j++) {
            const int q[3] = {k[0] + dx, k[1] + j / 3 - 1, k[2] + j % 3 - 1};
            in[j] = !(dx == 0 && j == 4) && q[0] >= -KEY_BIAS && q[0] <= KEY_BIAS - 1 && q[1] >= -KEY_BIAS &&
                    q[1] <= KEY_BIAS - 1 && q[2] >= -KEY_BIAS && q[2] <= KEY_BIAS - 1;
            nk[j] = ((unsigned long long)(q[0] + KEY_BIAS) << (2 * KEY_BITS)) |
                    ((unsigned long long)(q[1] + KEY_BIAS) << KEY_BITS) | (unsigned long long)(q[2] + KEY_BIAS);
            h[j] = mix64(nk[j]) & vt.mask;
            cur[j] = in[j] ? vt.keys[h[j]] : EMPTY_KEY;
        }
#pragma unroll
        for (int j = 0; j < 9; j++) {
            if (!in[j] || cur[j] == EMPTY_KEY) continue;
            const int nl = cur[j] == nk[j] ? vt.labels[h[j]] : vt_label(vt, nk[j]);
            if (nl < 0) continue;
            const int r = inst.parent[nl];
            bool seen = false;
            for (int t = 0; t < nr; t++) seen |= roots[t] == r;
            if (!seen) roots[nr++] = r;
        }
    }
    for (int j = 0; j < nr; j++) add_pair(sc, ss, ((unsigned long long)m << 32) | (unsigned)roots[j]);
}

__device__ void phase_overlap(const Scratch& sc, const SerialScratch& ss, const VoxelTable& vt, const Instances& inst,
                              unsigned char* smem, bool dilate)
{
    unsigned long long* pkey = (unsigned long long*)smem;   // [OV_SLOTS]
    int* pcnt = (int*)(pkey + OV_SLOTS);                    // [OV_SLOTS]
    constexpr int OV_THREADS = SER_THREADS;
    const int ne = sc.ctr->n_entries;
    if (blockIdx.x * OV_THREADS >= ne) return;  // no entries for this block (uniform)
    for (int i = threadIdx.x; i < OV_SLOTS; i += OV_THREADS) {
        pkey[i] = EMPTY_KEY;
        pcnt[i] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int i0 = blockIdx.x * OV_THREADS; i0 < ne; i0 += gridDim.x * OV_THREADS) {
        const int i = i0 + threadIdx.x;
        int new_slot = -1;  // slot of the new-voxel hash this thread claimed
        if (i < ne) {
            const unsigned long long hk = sc.sent[i];
            const int m = (int)(hk >> 54);
            const unsigned long long key = hk & ((1ull << 54) - 1);
            int lab = sc.elab[i];
            if (lab < 0) {
                // absent when the batch started: an earlier frame may have added it
                unsigned long long h = mix64(key) & vt.mask;
                for (int pr = 0;; pr++) {
                    const unsigned long long kk = vt.keys[h];
                    if (kk == key) { lab = vt.labels[h]; break; }
                    if (kk == EMPTY_KEY || pr > (int)vt.mask) break;
                    h = (h + 1) & vt.mask;
                }
            }
            if (dilate) dilated_pairs(sc, ss, vt, inst, m, key, lab);
            if (lab >= 0 && !dilate) {
                const unsigned long long okey = ((unsigned long long)m << 32) | (unsigned)inst.parent[lab];
                unsigned t = (unsigned)(mix64(okey) & (OV_SLOTS - 1));
                while (true) {
                    const unsigned long long prev = atomicCAS(&pkey[t], EMPTY_KEY, okey);
                    if (prev == EMPTY_KEY || prev == okey) break;
                    t = (t + 1) & (OV_SLOTS - 1);
                }
                atomicAdd(&pcnt[t], 1);
            } else if (lab < 0) {
                unsigned long long t = mix64(key) & ss.nmask;
                for (int pr = 0;; pr++) {
                    const unsigned long long cur = ss.nkeys[t];
                    if (cur == key) break;
                    if (cur == EMPTY_KEY) {
                        const unsigned long long prev = atomicCAS(&ss.nkeys[t], EMPTY_KEY, key);
                        if (prev == EMPTY_KEY) { new_slot = (int)t; break; }
                        if (prev == key) break;
                    }
                    t = (t + 1) & ss.nmask;
                    if (pr > (int)ss.nmask) { set_err(sc.ctr, DISC_ERR_TABLE_FULL); break; }
                }
                atomicMin(&ss.nown[t], m);
            }
        }
        // warp-aggregated append of the claimed new-voxel slots
        {
            const unsigned want = __ballot_sync(0xffffffffu, new_slot >= 0);
            int base = 0;
            if (lane == 0 && want) base = atomicAdd(&sc.ctr->n_new, __popc(want));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (new_slot >= 0) ss.nlist[base + __popc(want & ((1u << lane) - 1))] = new_slot;
        }
        __syncthreads();
        // flush the block's distinct pairs, then clear them for the next pass
        for (int j0 = 0; j0 < OV_SLOTS; j0 += OV_THREADS) {
            const int j = j0 + threadIdx.x;
            const unsigned long long okey = pkey[j];
            int pair_slot = -1;
            if (okey != EMPTY_KEY) {
                unsigned long long t = mix64(okey) & ss.omask;
                for (int pr = 0;; pr++) {
                    const unsigned long long cur = ss.okeys[t];
                    if (cur == okey) break;
                    if (cur == EMPTY_KEY) {
                        const unsigned long long prev = atomicCAS(&ss.okeys[t], EMPTY_KEY, okey);
                        if (prev == EMPTY_KEY) { pair_slot = (int)t; break; }
                        if (prev == okey) break;
                    }
                    t = (t + 1) & ss.omask;
                    if (pr > (int)ss.omask) { set_err(sc.ctr, DISC_ERR_TABLE_FULL); break; }
                }
                atomicAdd(&ss.ocnt[t], pcnt[j]);
                pkey[j] = EMPTY_KEY;
                pcnt[j] = 0;
            }
            const unsigned want = __ballot_sync(0xffffffffu, pair_slot >= 0);
            int base = 0;
            if (lane == 0 && want) base = atomicAdd(&sc.ctr->n_pairs, __popc(want));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (pair_slot >= 0) ss.olist[base + __popc(want & ((1u << lane) - 1))] = pair_slot;
        }
        __syncthreads();
    }
}

// ---- gates per (segment, instance) pair: one warp per pair -----------------------
// The fast cosine takes the tensor-core pooled embedding and the instance's
// scoring copy (fp32, bf16 at BF16 precision, E4M3 at FP8 precision: the
// copy's power-of-two scale cancels in the cosine); inside its error band the
// pair is re-scored exactly.
__device__ __forceinline__ unsigned bf16_pair(float lo, float hi)
{
    return (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
           ((unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

__device__ __forceinline__ float4 bf16x4_to_f32(uint2 v)
{
    return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u), __uint_as_float(v.y << 16),
                       __uint_as_float(v.y & 0xffff0000u));
}

// With a second grid (inst.A), the fast and exact features, their bounds and
// the instance side all come from the association features (view scratch va).
struct GateFeatures {
    const float* fast;    // [M][D] tensor-core pooled features
    const float* exact;   // [M][D] exact pooled features
    const float* bm;      // [M] sum_p w ||f_p|| (error-bound scale)
    const float* Sm;      // [cap][D] instances' scoring master
    int D;
};

__device__ __forceinline__ GateFeatures gate_features(const FrameParams& fp, const Scratch& sc, const Scratch& va,
                                                      const Instances& inst)
{
    GateFeatures g;
    g.D = scoring_dim(inst, fp.D);
    g.Sm = scoring_master(inst);
    g.fast = inst.A ? va.Efast : sc.Efast;
    g.exact = inst.A ? va.Ecan : sc.Ecan;
    g.bm = inst.A ? va.Bm : sc.Bm;
    return g;
}

// The cosine gate of segment m against instance k, by one warp (all 32 lanes
// call; every lane returns the decision).  The fast cosine takes the
// tensor-core pooled feature and the instance's scoring copy; inside its
// error band the pair is re-scored exactly (*border counts those).
__device__ bool warp_cosine_gate(const FrameParams& fp, const GateFeatures& gf, const Instances& inst, int m, int k,
                                 int* border)
{
    const int lane = threadIdx.x & 31;
    const int D = gf.D;
    const float* fast = gf.fast;
    const float* exact = gf.exact;
    const float* bm = gf.bm;
    const float* Sm = gf.Sm;
    const float* a = fast + (size_t)m * D;
    const float* b = Sm + (size_t)k * D;
    const float bmm = bm[m], erk = inst.Er ? inst.Er[k] : 0.0f;  // loaded beside the rows
    float dt = 0.0f, na = 0.0f, nb = 0.0f;
    if (inst.Eb && (D & 3) == 0) {  // bf16 scoring copy: 8-byte rows of 4
        const float4* a4 = (const float4*)a;
        const uint2* b4 = (const uint2*)(inst.Eb + (size_t)k * D);
        const int n4 = D >> 2;
        for (int d0 = 0; d0 < n4; d0 += 32 * 4) {
            float4 xs[4];
            uint2 ys[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int d = d0 + j * 32 + lane;
                xs[j] = d < n4 ? a4[d] : make_float4(0.f, 0.f, 0.f, 0.f);
                ys[j] = d < n4 ? b4[d] : make_uint2(0u, 0u);
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float4 x = xs[j], y = bf16x4_to_f32(ys[j]);
                dt += x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
                na += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
                nb += y.x * y.x + y.y * y.y + y.z * y.z + y.w * y.w;
            }
        }
    } else if (inst.E8 && (D & 3) == 0) {  // E4M3 scoring copy: 4-byte words of 4
        const float4* a4 = (const float4*)a;
        const uint32_t* b4 = (const uint32_t*)(inst.E8 + (size_t)k * D);
        const int n4 = D >> 2;
        for (int d0 = 0; d0 < n4; d0 += 32 * 4) {
            float4 xs[4];
            uint32_t ys[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int d = d0 + j * 32 + lane;
                xs[j] = d < n4 ? a4[d] : make_float4(0.f, 0.f, 0.f, 0.f);
                ys[j] = d < n4 ? b4[d] : 0u;
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float4 x = xs[j];
                const float y0 = from_e4m3(ys[j] & 0xffu), y1 = from_e4m3((ys[j] >> 8) & 0xffu);
                const float y2 = from_e4m3((ys[j] >> 16) & 0xffu), y3 = from_e4m3(ys[j] >> 24);
                dt += x.x * y0 + x.y * y1 + x.z * y2 + x.w * y3;
                na += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
                nb += y0 * y0 + y1 * y1 + y2 * y2 + y3 * y3;
            }
        }
    } else if (inst.E8) {
        const uint8_t* b8 = inst.E8 + (size_t)k * D;
        for (int d = lane; d < D; d += 32) {
            const float x = a[d], y = from_e4m3(b8[d]);
            dt += x * y;
            na += x * x;
            nb += y * y;
        }
    } else if (inst.Eb) {
        const uint16_t* bb = inst.Eb + (size_t)k * D;
        for (int d = lane; d < D; d += 32) {
            const float x = a[d], y = __uint_as_float((unsigned)bb[d] << 16);
            dt += x * y;
            na += x * x;
            nb += y * y;
        }
    } else if ((D & 3) == 0 && D <= 1024) {  // 16-byte rows of up to 1024: every load in flight at once
        const float4* a4 = (const float4*)a;
        const float4* b4 = (const float4*)b;
        const int n4 = D >> 2;
        float4 xs[8], ys[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int d = j * 32 + lane;
            xs[j] = d < n4 ? a4[d] : make_float4(0.f, 0.f, 0.f, 0.f);
            ys[j] = d < n4 ? b4[d] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const float4 x = xs[j], y = ys[j];
            dt += x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
            na += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
            nb += y.x * y.x + y.y * y.y + y.z * y.z + y.w * y.w;
        }
    } else if ((D & 3) == 0) {  // rows are 16-byte aligned: vector loads, 8 in flight per lane
        const float4* a4 = (const float4*)a;
        const float4* b4 = (const float4*)b;
        const int n4 = D >> 2;
        for (int d0 = 0; d0 < n4; d0 += 32 * 4) {
            float4 xs[4], ys[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int d = d0 + j * 32 + lane;
                xs[j] = d < n4 ? a4[d] : make_float4(0.f, 0.f, 0.f, 0.f);
                ys[j] = d < n4 ? b4[d] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float4 x = xs[j], y = ys[j];
                dt += x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
                na += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
                nb += y.x * y.x + y.y * y.y + y.z * y.z + y.w * y.w;
            }
        }
    } else {
        for (int d = lane; d < D; d += 32) {
            const float x = a[d], y = b[d];
            dt += x * y;
            na += x * x;
            nb += y * y;
        }
    }
    dt = warp_sum(dt);
    na = warp_sum(na);
    nb = warp_sum(nb);
    bool edge;
    const float cf = (na > 0.0f && nb > 0.0f) ? dt / (sqrtf(na) * sqrtf(nb)) : 0.0f;
    // |cos(a, b') - cos(e, b)| <= 2 |a - e| / |a| + 2 |b' - b| / |b|, plus
    // the fp32 arithmetic of cf; 10 % slack on the bounds
    float band = (na > 0.0f) ? 2.2f * fp.eta * bmm / sqrtf(na) + fp.dot_err + 1e-6f : 2.0f;
    if (inst.Er) band += 2.2f * erk;
    if (fabsf(cf - fp.tau) > band) {
        edge = cf >= fp.tau;
    } else {
        // exact re-score with the exact pooled embedding
        const float* ae = exact + (size_t)m * D;
        long long xd = 0, xa = 0, xb = 0;
        if ((D & 3) == 0) {  // all of a lane's loads in flight before the exact sums
            const float4* a4 = (const float4*)ae;
            const float4* b4 = (const float4*)b;
            const int n4 = D >> 2;
            for (int d0 = 0; d0 < n4; d0 += 32 * 4) {
                float4 xs[4], ys[4];
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int d = d0 + j * 32 + lane;
                    xs[j] = d < n4 ? a4[d] : make_float4(0.f, 0.f, 0.f, 0.f);
                    ys[j] = d < n4 ? b4[d] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const float xv[4] = {xs[j].x, xs[j].y, xs[j].z, xs[j].w};
                    const float yv[4] = {ys[j].x, ys[j].y, ys[j].z, ys[j].w};
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        xd += fix32f(__fmul_rn(xv[c], yv[c]), S_SQ);
                        xa += fix32f(__fmul_rn(xv[c], xv[c]), S_SQ);
                        xb += fix32f(__fmul_rn(yv[c], yv[c]), S_SQ);
                    }
                }
            }
        } else {
            for (int d = lane; d < D; d += 32) {
                const float x = ae[d], y = b[d];
                xd += fix32f(__fmul_rn(x, y), S_SQ);
                xa += fix32f(__fmul_rn(x, x), S_SQ);
                xb += fix32f(__fmul_rn(y, y), S_SQ);
            }
        }
        xd = warp_sum(xd);
        xa = warp_sum(xa);
        xb = warp_sum(xb);
        float ce = 0.0f;
        if (xa != 0 && xb != 0)
            ce = __double2float_rn(__ddiv_rn(unfix(xd, S_SQ),
                                             __dmul_rn(__dsqrt_rn(unfix(xa, S_SQ)), __dsqrt_rn(unfix(xb, S_SQ)))));
        edge = ce >= fp.tau;
        (*border)++;
    }
    return edge;
}

// Warps w0, w0 + nw, ... of the launch take the pairs in turn.
__device__ void phase_score(const FrameParams& fp, const Scratch& sc, const Scratch& va, const SerialScratch& ss,
                            const Instances& inst, int w0, int nw)
{
    const int lane = threadIdx.x & 31;
    const int npairs = sc.ctr->n_pairs;
    const GateFeatures gf = gate_features(fp, sc, va, inst);
    int border = 0, scored = 0;
    for (int i = w0; i < npairs; i += nw) {
        const int slot = ss.olist[i];
        const unsigned long long okey = ss.okeys[slot];
        const int m = (int)(okey >> 32) - 1;
        const int k = (int)(okey & 0xffffffffu);
        const long long ov = ss.ocnt[slot];
        // overlap coefficient |V_m & V_k| / min(|V_m|, |V_k|) >= ov_num / ov_den
        const long long denom = min((long long)sc.nvox[m], inst.count[k]);
        if (ov * (long long)fp.ov_den < (long long)fp.ov_num * denom) continue;
        scored++;
        const bool edge = warp_cosine_gate(fp, gf, inst, m, k, &border);
        if (edge && lane == 0) {
            const int e = atomicAdd(ss.edge_n, 1);
            if (e < ss.edge_cap) {
                ss.edge_m[e] = m;
                ss.edge_k[e] = k;
            } else {
                set_err(sc.ctr, DISC_ERR_CAPACITY);
            }
        }
    }
    if (lane == 0 && border) atomicAdd(&sc.ctr->borderline, border);
    if (lane == 0 && scored) atomicAdd(&sc.ctr->n_scored, scored);
}

// ---- union, new ids, merges, fusion (one block) ------------------------------------
// Shared memory: a hash set of the frame's active roots (all overlap pairs)
// that also hands out local indices to the roots that carry an edge, and
// per-local-root arrays for the union-find and the fusion.  Every step runs
// in parallel on shared memory.  Any block of a multiple of 32 threads, at
// least MAX_MASKS, runs it.
constexpr int UNION_THREADS = 256;
constexpr int PAIR_CAP = 8192;             // distinct (segment, instance) overlaps per frame
constexpr int EDGE_ROOT_CAP = 2048;        // distinct instances with an accepted edge per frame
constexpr int EDGE_CAP = 4096;             // accepted (segment, instance) edges per frame
constexpr int UHASH = 2 * PAIR_CAP;        // hash slots at most (load <= 1/2); a frame uses
                                           // the next power of two >= 2 * its pairs
constexpr unsigned UH_EMPTY = 0xffffffffu;
constexpr unsigned UH_UNUSED = 0xffffffffu;
constexpr unsigned UH_LOCAL = 0x80000000u;
constexpr size_t UNION_SMEM = (size_t)UHASH * 8 + (size_t)EDGE_ROOT_CAP * 24 + (size_t)EDGE_CAP * 8;
static_assert(UNION_SMEM == (size_t)UHASH * 8 + (size_t)EDGE_ROOT_CAP * 24 + (size_t)EDGE_CAP * 8, "union layout");

// slot of root id k in the union's root hash (32-bit multiplicative mix)
__device__ __forceinline__ unsigned uhash(unsigned k, unsigned mask)
{
    unsigned h = k * 0x9E3779B1u;
    h ^= h >> 15;
    return h & mask;
}

// float <-> unsigned key with the same order (for atomicMax over floats)
__device__ __forceinline__ unsigned f2key(float x)
{
    const unsigned b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key2f(unsigned k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__device__ __forceinline__ int uf_find(const int* uf, int x)
{
    while (true) {
        const int p = ((volatile const int*)uf)[x];
        if (p == x) return x;
        x = p;
    }
}

__device__ __forceinline__ int local_of(const unsigned* hkey, const unsigned* hval, unsigned mask, unsigned k)
{
    unsigned h = uhash(k, mask);
    while (hkey[h] != k) h = (h + 1) & mask;
    return (int)(hval[h] & ~UH_LOCAL);
}

// Bytes of a union region with the given capacities (layout in
// UnionRegion); pre: with the arrays of values gathered before the union.
__host__ __device__ constexpr size_t union_region_bytes(unsigned uhash_cap, int root_cap, int edge_cap,
                                                        bool pre = false)
{
    return (size_t)uhash_cap * 8 + (size_t)root_cap * (pre ? 32 : 24) + (size_t)edge_cap * (pre ? 24 : 8);
}

// The arrays of a union region: the root hash, the per-local-root arrays
// and the edge arrays; with `pre` also each local root's voxel count (cloc)
// and, per edge, its instance's count, Q and observations as the gates read
// them (ec, eq, eo), so the union issues no global load for them.
struct UnionRegion {
    unsigned* hkey;      // [uhash_cap] root id
    unsigned* hval;      // [uhash_cap] claimant edge, then UH_LOCAL | local index
    long long* cloc;     // [root_cap] voxel count of the local roots (pre)
    int* gid;            // [root_cap] local -> instance id
    int* uf;             // union-find over local indices
    int* best_src;       // fusion winner per component
    float* best_q;
    float* qloc;         // Q of the local roots
    int* oloc;           // observations of the local roots
    long long* ec;       // [edge_cap] count of the edge's instance (pre)
    int* em;             // [edge_cap] edge segment
    int* ek;             // [edge_cap] edge instance id
    float* eq;           // [edge_cap] Q of the edge's instance (pre)
    int* eo;             // [edge_cap] observations of the edge's instance (pre)
    __device__ __forceinline__ UnionRegion(unsigned char* base, unsigned uhash_cap, int root_cap, int edge_cap,
                                           bool pre)
    {
        hkey = (unsigned*)base;
        hval = hkey + uhash_cap;
        cloc = pre ? (long long*)(hval + uhash_cap) : nullptr;
        gid = pre ? (int*)(cloc + root_cap) : (int*)(hval + uhash_cap);
        uf = gid + root_cap;
        best_src = uf + root_cap;
        best_q = (float*)(best_src + root_cap);
        qloc = best_q + root_cap;
        oloc = (int*)(qloc + root_cap);
        ec = pre ? (long long*)(oloc + root_cap) : nullptr;
        em = pre ? (int*)(ec + edge_cap) : oloc + root_cap;
        ek = em + edge_cap;
        eq = pre ? (float*)(ek + edge_cap) : nullptr;
        eo = pre ? (int*)(eq + edge_cap) : nullptr;
    }
};

// Per-segment inputs of the union read by the calling thread before the
// union starts (thread t for segment t; the frame's M <= block size), and
// what the union hands back to every thread when it completes.
struct UnionPre {
    int nv;       // nvox[t]
    float q;      // the segment's Q
    int nnew;     // voxels the frame inserts with segment t as their lowest segment
    int next;     // the map's next instance id
    int ok;       // out: the union completed without error
    int ncopy;    // out: embedding copies it listed
    int merges;   // out: instances it merged
};

// The frame's npairs overlap pairs give their roots through pair_root(i);
// its nedge accepted edges are in ss.edge_m/k, or (edges_in_place) already in
// the region's em/ek arrays (and, with pre, their instances' values in
// ec/eq/eo).  The region (shared memory, or global memory for frames beyond
// the shared capacities) is laid out as UnionRegion: hkey, hval [uhash_cap
// >= 2 * npairs], the per-root arrays [root_cap], the edge arrays [edge_cap
// >= 2 * root_cap: the fusion step lays root_cap 64-bit words over em].
// pre: the calling thread's per-segment values, read before the union; the
// union then also adds the frame's new voxels to their instances' counts.
// Past a capacity the frame fails with DISC_ERR_CAPACITY, or, soft, the
// call returns false before anything outside the region changed (the caller
// then retries with larger capacities); otherwise it returns true.
template <class PairRoot>
__device__ bool union_frame(const FrameParams& fp, const Scratch& sc, const SerialScratch& ss, const Instances& inst,
                            int* next_id, unsigned char* union_smem, unsigned uhash_cap, int root_cap, int edge_cap,
                            bool soft, int npairs, int nedge, bool edges_in_place, PairRoot pair_root,
                            UnionPre* pre = nullptr)
{
    const UnionRegion U(union_smem, uhash_cap, root_cap, edge_cap, pre != nullptr);
    unsigned* hkey = U.hkey;
    unsigned* hval = U.hval;
    int* gid = U.gid;
    int* uf = U.uf;
    int* best_src = U.best_src;
    float* best_q = U.best_q;
    float* qloc = U.qloc;
    int* oloc = U.oloc;
    int* em = U.em;
    int* ek = U.ek;
    __shared__ int anchor[MAX_MASKS];                 // smallest local root of a segment's edges
    __shared__ int srep[MAX_MASKS];
    __shared__ int snv[MAX_MASKS];
    __shared__ float sq[MAX_MASKS];
    __shared__ int s_nroots, s_nloc, s_merges, s_new, s_ncopy, s_next;
    const int tid = threadIdx.x, NT = blockDim.x;
    FrameCounters* ctr = sc.ctr;
    const int M = fp.M;
    if (2u * (unsigned)npairs > uhash_cap || nedge > edge_cap) {
        if (soft) return false;
        if (tid == 0) set_err(ctr, DISC_ERR_CAPACITY);
        return true;
    }
    unsigned hsize = 64;
    while (hsize < 2u * (unsigned)npairs) hsize <<= 1;
    const unsigned hm = hsize - 1;
    // the edges, once, into shared memory (segment, root)
    for (int e = tid; e < nedge && !edges_in_place; e += NT) {
        em[e] = ss.edge_m[e];
        ek[e] = ss.edge_k[e];
    }
    for (int i = tid; i < (int)hsize; i += NT) {
        hkey[i] = UH_EMPTY;
        hval[i] = UH_UNUSED;
    }
    if (pre) {
        if (tid < M) {
            anchor[tid] = INT_MAX;
            snv[tid] = pre->nv;
            sq[tid] = pre->q;
        }
    } else {
        for (int m = tid; m < M; m += NT) {
            anchor[m] = INT_MAX;
            snv[m] = sc.nvox[m];
            sq[m] = sc.S[5 * m + 4];
        }
    }
    if (tid == 0) {
        s_nroots = 0;
        s_nloc = 0;
        s_merges = 0;
        s_new = 0;
        s_ncopy = 0;
        s_next = pre ? pre->next : *next_id;
    }
    __syncthreads();
    // (1) active set: distinct roots of all overlap pairs (counted per warp)
    {
        int mine = 0;
        for (int i = tid; i < npairs; i += NT) {
            const unsigned k = pair_root(i);
            unsigned h = uhash(k, hm);
            while (true) {
                const unsigned cur = hkey[h];
                if (cur == k) break;
                if (cur == UH_EMPTY) {
                    const unsigned prev = atomicCAS(&hkey[h], UH_EMPTY, k);
                    if (prev == UH_EMPTY) { mine++; break; }
                    if (prev == k) break;
                }
                h = (h + 1) & hm;
            }
        }
        mine = warp_sum(mine);
        if ((tid & 31) == 0 && mine) atomicAdd(&s_nroots, mine);
    }
    __syncthreads();
    // (2) local indices for the roots that carry an edge: the first edge to
    //     claim a root's slot assigns the index
    for (int e = tid; e < nedge; e += NT) {
        const unsigned k = (unsigned)ek[e];
        unsigned h = uhash(k, hm);
        while (hkey[h] != k) h = (h + 1) & hm;
        atomicCAS(&hval[h], UH_UNUSED, (unsigned)e);
    }
    __syncthreads();
    for (int e = tid; e < nedge; e += NT) {
        const unsigned k = (unsigned)ek[e];
        unsigned h = uhash(k, hm);
        while (hkey[h] != k) h = (h + 1) & hm;
        if (hval[h] == (unsigned)e) {
            const int x = atomicAdd(&s_nloc, 1);
            if (x < root_cap) {
                gid[x] = (int)k;
                uf[x] = x;
                if (pre) {
                    qloc[x] = U.eq[e];
                    oloc[x] = U.eo[e];
                    U.cloc[x] = U.ec[e];
                } else {
                    qloc[x] = inst.Q[k];
                    oloc[x] = inst.n_obs[k];
                }
            }
            hval[h] = UH_LOCAL | (unsigned)x;
        }
    }
    __syncthreads();
    const int nloc = s_nloc;
    if (nloc > root_cap) {
        if (soft) return false;
        if (tid == 0) set_err(ctr, DISC_ERR_CAPACITY);
        return true;
    }
    // (3) union of the instances one segment joins: every edge hooks its
    //     root onto the segment's anchor; a hook always links the root with
    //     the larger instance id under the smaller one, so each set's root is
    //     its smallest instance id
    for (int e = tid; e < nedge; e += NT) atomicMin(&anchor[em[e]], local_of(hkey, hval, hm, (unsigned)ek[e]));
    __syncthreads();
    for (int e = tid; e < nedge; e += NT) {
        int x = local_of(hkey, hval, hm, (unsigned)ek[e]);
        int y = anchor[em[e]];
        while (true) {
            x = uf_find(uf, x);
            y = uf_find(uf, y);
            if (x == y) break;
            const int lo = gid[x] < gid[y] ? x : y, hi = lo == x ? y : x;
            if (atomicCAS(&uf[hi], hi, lo) == hi) break;
        }
    }
    __syncthreads();
    for (int x = tid; x < nloc; x += NT) uf[x] = uf_find(uf, x);  // stores only roots
    __syncthreads();
    for (int m = tid; m < M; m += NT) srep[m] = anchor[m] != INT_MAX ? gid[uf[anchor[m]]] : -1;
    __syncthreads();
    // (4) new instances for live segments without an edge, in mask order:
    //     the id of mask m is next_id plus the number of such masks before it
    //     (a block-wide exclusive scan; M <= MAX_MASKS <= NT)
    {
        __shared__ int wtot[32];
        const int lane = tid & 31, wid = tid >> 5;
        const bool want = tid < M && snv[tid] > 0 && srep[tid] < 0;
        const unsigned bal = __ballot_sync(0xffffffffu, want);
        if (lane == 0) wtot[wid] = __popc(bal);
        __syncthreads();
        int before = __popc(bal & ((1u << lane) - 1)), total = 0;
        for (int w = 0; w < (NT >> 5); w++) {
            before += w < wid ? wtot[w] : 0;
            total += wtot[w];
        }
        const int base = s_next;
        if (base + total > inst.cap) {  // uniform: every thread summed the same counts
            if (tid == 0) set_err(ctr, DISC_ERR_CAPACITY);
            return true;
        }
        if (want) {
            const int id = base + before, m = tid;
            srep[m] = id;
            inst.parent[id] = id;
            inst.count[id] = 0;
            inst.Q[id] = sq[m];
            inst.n_obs[id] = 1;
            ss.copy_dst[before] = id;
            ss.copy_src[before] = -(m + 1);
        }
        __syncthreads();  // every thread has read s_next
        if (tid == 0) {
            *next_id = base + total;
            s_next = base + total;
            s_new = total;
            s_ncopy = total;
        }
    }
    __syncthreads();
    for (int m = tid; m < M; m += NT) sc.segrep[m] = srep[m];
    // (5) fusion per component: the candidates in the order (members by
    //     ascending id, then segments by ascending mask) keep the first one
    //     whose Q is the component's maximum (strict '>' while scanning):
    //     the component's maximum (an atomic max on order-preserving keys),
    //     then the smallest member id with that Q, else the smallest mask;
    //     the stored Q is the winner's own value.  The edge arrays are no
    //     longer needed and hold part of the per-root scratch.
    unsigned* qmax = (unsigned*)best_q;                              // [nloc] key of the max Q
    int* obs = best_src;                                             // [nloc] observations
    unsigned long long* src_inst = (unsigned long long*)em;          // [nloc] (id << 32 | local) at the max
    int* src_seg = ek;                                               // [nloc] smallest mask at the max
    for (int r = tid; r < nloc; r += NT) {
        qmax[r] = 0u;
        obs[r] = 0;
        src_inst[r] = ~0ull;
        src_seg[r] = INT_MAX;
    }
    // the local root of each segment that joined a component
    for (int m = tid; m < M; m += NT) snv[m] = anchor[m] != INT_MAX ? uf[anchor[m]] : -1;
    __syncthreads();
    for (int x = tid; x < nloc; x += NT) {
        atomicMax(&qmax[uf[x]], f2key(qloc[x]));
        atomicAdd(&obs[uf[x]], oloc[x]);
    }
    for (int m = tid; m < M; m += NT)
        if (snv[m] >= 0) {
            atomicMax(&qmax[snv[m]], f2key(sq[m]));
            atomicAdd(&obs[snv[m]], 1);
        }
    __syncthreads();
    for (int x = tid; x < nloc; x += NT)
        if (qloc[x] == key2f(qmax[uf[x]]))
            atomicMin(&src_inst[uf[x]], ((unsigned long long)(unsigned)gid[x] << 32) | (unsigned)x);
    for (int m = tid; m < M; m += NT)
        if (snv[m] >= 0 && sq[m] == key2f(qmax[snv[m]])) atomicMin(&src_seg[snv[m]], m);
    __syncthreads();
    for (int r = tid; r < nloc; r += NT) {
        if (uf[r] != r) continue;
        const int rep = gid[r];
        inst.n_obs[rep] = obs[r];
        int src;
        float q;
        if (src_inst[r] != ~0ull) {
            const int x = (int)(src_inst[r] & 0xffffffffu);
            src = gid[x];
            q = qloc[x];
        } else {
            src = -(src_seg[r] + 1);
            q = sq[src_seg[r]];
        }
        if (src == rep) continue;
        const int c = atomicAdd(&s_ncopy, 1);
        ss.copy_dst[c] = rep;
        ss.copy_src[c] = src;
        inst.Q[rep] = q;
    }
    // (6) merge members into their representative (then, with pre, the
    //     frame's new voxels into their segment's instance)
    for (int x = tid; x < nloc; x += NT) {
        const int r = uf[x];
        if (r == x) continue;
        const int k = gid[x], rep = gid[r];
        inst.parent[k] = rep;
        atomicAdd((unsigned long long*)&inst.count[rep], (unsigned long long)(pre ? U.cloc[x] : inst.count[k]));
        inst.count[k] = 0;
        atomicAdd(&s_merges, 1);
    }
    if (pre && tid < M && pre->nnew && srep[tid] >= 0)
        atomicAdd((unsigned long long*)&inst.count[srep[tid]], (unsigned long long)pre->nnew);
    __syncthreads();
    if (tid == 0) {
        *ss.copy_n = s_ncopy;
        *ss.edge_n = 0;  // the next frame's gates start a new edge list
        ctr->active_instances = s_nroots;
        ctr->new_instances = s_new;
        ctr->merges = s_merges;
        ctr->n_edges = nedge;
        ctr->next_id = s_next;
        ctr->n_copies = s_ncopy;
    }
    if (pre) {
        pre->ok = 1;
        pre->ncopy = s_ncopy;
        pre->merges = s_merges;
    }
    return true;
}

// The frame's pairs in the map's global pair hash, its edges in ss.edge_m/k;
// union_smem: a region of UNION_SMEM bytes (shared or global memory).
__device__ void phase_union(const FrameParams& fp, const Scratch& sc, const SerialScratch& ss, const Instances& inst,
                            int* next_id, unsigned char* union_smem)
{
    const int npairs = sc.ctr->n_pairs;
    const int nedge = min(*ss.edge_n, ss.edge_cap);
    union_frame(fp, sc, ss, inst, next_id, union_smem, UHASH, EDGE_ROOT_CAP, EDGE_CAP, false, npairs, nedge, false,
                [&](int i) { return (unsigned)(ss.okeys[ss.olist[i]] & 0xffffffffu); });
}

// One warp copies an embedding row (and writes its bf16 copy when tb is set).
__device__ __forceinline__ void copy_row(const float* from, float* to, uint16_t* tb, int D, int lane)
{
    if ((D & 3) == 0) {
        const float4* f4 = (const float4*)from;
        float4* t4 = (float4*)to;
        const int n4 = D >> 2;
        for (int d0 = 0; d0 < n4; d0 += 32 * 8) {
            float4 r[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int d = d0 + j * 32 + lane;
                if (d < n4) r[j] = f4[d];
            }
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int d = d0 + j * 32 + lane;
                if (d < n4) {
                    t4[d] = r[j];
                    if (tb) ((uint2*)tb)[d] = make_uint2(bf16_pair(r[j].x, r[j].y), bf16_pair(r[j].z, r[j].w));
                }
            }
        }
    } else {
        for (int d = lane; d < D; d += 32) {
            to[d] = from[d];
            if (tb) tb[d] = __bfloat16_as_ushort(__float2bfloat16_rn(from[d]));
        }
    }
}

// ---- embeddings, new voxels, parent flattening, cleanup ---------------------------
__device__ void phase_apply(const FrameParams& fp, const Scratch& sc, const Scratch& va, const SerialScratch& ss,
                            const VoxelTable& vt,
                            const Instances& inst, const int* next_id, bool ok)
{
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gsz = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int D = fp.D;
    if (ok) {
        // winning embeddings (the sources are never written in this frame):
        // one warp per vector, all loads in flight before the stores; the
        // scoring copies follow the scoring master (the association feature
        // with a second grid)
        const int nc = *ss.copy_n;
        for (int c = gtid >> 5; c < nc; c += gsz >> 5) {
            const int src = ss.copy_src[c], dst = ss.copy_dst[c];
            const float* from = src >= 0 ? inst.E + (size_t)src * D : sc.Ecan + (size_t)(-src - 1) * D;
            if (inst.A) {
                const int Da = inst.Da;
                const float* fa = src >= 0 ? inst.A + (size_t)src * Da : va.Ecan + (size_t)(-src - 1) * Da;
                copy_row(from, inst.E + (size_t)dst * D, nullptr, D, lane);
                copy_row(fa, inst.A + (size_t)dst * Da, inst.Eb ? inst.Eb + (size_t)dst * Da : nullptr, Da, lane);
                if (inst.E8) e4m3_copy_row(fa, Da, inst.E8 + (size_t)dst * Da, inst.Er + dst);
            } else {
                copy_row(from, inst.E + (size_t)dst * D, inst.Eb ? inst.Eb + (size_t)dst * D : nullptr, D, lane);
                if (inst.E8) e4m3_copy_row(from, D, inst.E8 + (size_t)dst * D, inst.Er + dst);
            }
        }
        // new voxels: the lowest segment index owns a voxel
        const int nn = sc.ctr->n_new;
        for (int i = gtid; i < nn; i += gsz) {
            const int t = ss.nlist[i];
            const unsigned long long key = ss.nkeys[t];
            const int lab = sc.segrep[ss.nown[t] - 1];
            unsigned long long h = mix64(key) & vt.mask;
            for (int pr = 0;; pr++) {
                const unsigned long long prev = atomicCAS(&vt.keys[h], EMPTY_KEY, key);
                if (prev == EMPTY_KEY) { vt.labels[h] = lab; break; }
                h = (h + 1) & vt.mask;
                if (pr > (int)vt.mask) { set_err(sc.ctr, DISC_ERR_TABLE_FULL); break; }
            }
            // one count update per distinct instance of the warp
            const unsigned grp = __match_any_sync(__activemask(), lab);
            if (lane == __ffs(grp) - 1) atomicAdd((unsigned long long*)&inst.count[lab], (unsigned long long)__popc(grp));
        }
        if (gtid == 0) atomicAdd(vt.used, (unsigned long long)nn);
        // keep the parent table flat (two levels at most after this frame)
        if (sc.ctr->merges > 0) {
            const int nid = *next_id;
            for (int i = gtid; i < nid; i += gsz) inst.parent[i] = inst.parent[inst.parent[i]];
        }
    }
    // cleanup of the serial hashes, whatever happened above
    const int np = sc.ctr->n_pairs, nn = sc.ctr->n_new;
    for (int i = gtid; i < np; i += gsz) {
        const int s = ss.olist[i];
        ss.okeys[s] = EMPTY_KEY;
        ss.ocnt[s] = 0;
    }
    for (int i = gtid; i < nn; i += gsz) {
        const int s = ss.nlist[i];
        // inserted above before this thread reset it: same thread, same i
        ss.nkeys[s] = EMPTY_KEY;
        ss.nown[s] = INT_MAX;
    }
}

// ---- kernels ------------------------------------------------------------------------
// Block row g runs frame j of map g.  Whether the frame is blocked is decided
// once per block (another block may raise an error while this one reads), so
// every thread of the block takes the same path.  Returns the frame slot, or
// -1 when map g has no frame j or the frame is blocked.
// The frame slot of this block's map (block row g) and whether the frame is
// blocked: by its own error, or (full check, the frame's first serial kernel)
// by an error of the map's previous frame, which is then copied into this
// frame's counters so that its later kernels need only their own.  Warp 0
// loads the slot indices side by side, then both status words: two round
// trips before the block's barrier.
__device__ int block_slot(const BatchScratch& bs, const SerialStep& st, bool* blocked, bool full)
{
    __shared__ int s_slot, s_blocked;
    const int g = blockIdx.y;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const bool prev_in_batch = st.j > 0;
        int v = -1;
        if (lane == 0)
            v = st.slot_of[g * st.J + st.j];
        else if (lane == 1 && full)
            v = prev_in_batch ? st.slot_of[g * st.J + st.j - 1] : st.prev_hist[g];
        const int slot = __shfl_sync(0xffffffffu, v, 0);
        const int pidx = __shfl_sync(0xffffffffu, v, 1);
        int e = 0;
        if (lane == 0 && slot >= 0)
            e = bs.frame(slot).ctr->err;
        else if (lane == 1 && full && pidx >= 0)
            e = prev_in_batch ? bs.frame(pidx).ctr->err : st.hist[pidx].err;
        const int own = __shfl_sync(0xffffffffu, e, 0);
        const int prev = __shfl_sync(0xffffffffu, e, 1);
        if (lane == 0) {
            bool b = slot >= 0 && own != 0;
            if (slot >= 0 && !b && full && prev) {
                set_err(bs.frame(slot).ctr, prev);
                b = true;
            }
            s_slot = slot;
            s_blocked = b ? 1 : 0;
        }
    }
    __syncthreads();
    const int slot = s_slot;
    *blocked = s_blocked != 0;
    __syncthreads();
    return slot;
}

constexpr size_t OV_SMEM = (size_t)OV_SLOTS * 12;

__global__ void __launch_bounds__(SER_THREADS) k_overlap(const FrameParams* fps, BatchScratch bs, SerialStep st)
{
    extern __shared__ __align__(16) unsigned char ov_smem[];
    bool blocked;
    const int slot = block_slot(bs, st, &blocked, true);
    if (slot < 0 || blocked) return;
    const MapRefs& R = st.refs[blockIdx.y];
    const SerialScratch ss = R.ss;
    const VoxelTable vt = R.vt;
    const Instances inst = R.inst;
    phase_overlap(bs.frame(slot), ss, vt, inst, ov_smem, fps[slot].dilate != 0);
}

__global__ void k_score(const FrameParams* fps, BatchScratch bs, SerialStep st)
{
    bool blocked;
    const int slot = block_slot(bs, st, &blocked, false);
    if (slot < 0 || blocked) return;
    const MapRefs& R = st.refs[blockIdx.y];
    const SerialScratch ss = R.ss;
    const Instances inst = R.inst;
    phase_score(fps[slot], bs.frame(slot), st.view.frame(slot), ss, inst, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                (gridDim.x * blockDim.x) >> 5);
}

__global__ void __launch_bounds__(UNION_THREADS, 1) k_union(const FrameParams* fps, BatchScratch bs, SerialStep st)
{
    extern __shared__ __align__(16) unsigned char union_smem[];
    bool blocked;
    const int slot = block_slot(bs, st, &blocked, false);
    if (slot < 0 || blocked) return;
    const MapRefs& R = st.refs[blockIdx.y];
    const SerialScratch ss = R.ss;
    const Instances inst = R.inst;
    phase_union(fps[slot], bs.frame(slot), ss, inst, R.next_id, union_smem);
}

__global__ void k_apply(const FrameParams* fps, BatchScratch bs, SerialStep st)
{
    bool blocked;
    const int slot = block_slot(bs, st, &blocked, false);
    if (slot < 0) return;
    const MapRefs& R = st.refs[blockIdx.y];
    const SerialScratch ss = R.ss;
    const VoxelTable vt = R.vt;
    const Instances inst = R.inst;
    phase_apply(fps[slot], bs.frame(slot), st.view.frame(slot), ss, vt, inst, R.next_id, !blocked);
}

__global__ void k_serial_begin(const MapRefs* refs, int G)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < G) {
        *refs[g].ss.edge_n = 0;
        *refs[g].ss.copy_n = 0;
    }
}

// ==== The frame chain as one pass per batch ==========================================
// The overlap histogram of frame j (Sec. III-B) counts, per segment m and
// instance root k, the segment's voxels whose label resolves to k in the map
// as frame j finds it.  A voxel of frame j is either
//   (a) in the map when the batch starts: its label is known before any frame
//       of the batch runs, only its root may change as earlier frames merge;
//   (b) absent then, and first seen in this batch by an earlier frame j0 of
//       the same map: that frame inserts it with the instance its lowest
//       segment m0 joins (Sec. III-B, reading O11), known once frame j0 is
//       associated;
//   (c) absent until frame j itself: a new voxel of frame j (no overlap),
//       owned by its lowest segment.
// So the per-voxel work of the whole batch runs before the frames run in
// order: k_lookup probes every (segment, voxel) entry of every frame in the
// map as it stands at the batch start and gathers each absent voxel's first
// (frame, segment) of the batch in one batch-wide hash; k_absent sorts the
// absent entries into (b) and (c).  Each frame is left with a few hundred
// to a few thousand items, (m, label) and (m, j0, m0), with voxel counts.
// k_associate then runs each map's frames in order in one CTA (overlap pairs
// from the items, the gates, the union, fusion and the voxel counts), and
// k_commit inserts the batch's new voxels with their first frame's labels and
// flattens the parent tables.  A frame that fails inserts nothing, and the
// frames after it in its map are blocked.

constexpr unsigned long long KEY54 = (1ull << 54) - 1;

// The warp's lanes with `want` set add one voxel each to overlap item `key`
// of the frame: lanes with the same key add together (one atomic per
// distinct key of the warp).  All 32 lanes call.
__device__ __forceinline__ void add_item_warp(const Scratch& sc, unsigned long long key, bool want)
{
    const unsigned act = __ballot_sync(0xffffffffu, want);
    if (!want) return;
    const unsigned grp = __match_any_sync(act, key);
    if ((int)(threadIdx.x & 31) != __ffs(grp) - 1) return;
    unsigned long long t = mix64(key) & sc.smask;
    for (unsigned long long pr = 0;; pr++) {
        const unsigned long long cur = sc.pkey[t];
        if (cur == key) break;
        if (cur == EMPTY_KEY) {
            const unsigned long long prev = atomicCAS(&sc.pkey[t], EMPTY_KEY, key);
            if (prev == EMPTY_KEY) {
                sc.plist[atomicAdd(&sc.ctr->n_pre, 1)] = (int)t;
                break;
            }
            if (prev == key) break;
        }
        t = (t + 1) & sc.smask;
        if (pr > sc.smask) {
            set_err(sc.ctr, DISC_ERR_TABLE_FULL);
            return;
        }
    }
    atomicAdd(&sc.pcnt[t], __popc(grp));
}

// Warp-aggregated append: each lane with `want` gets a distinct index from
// the counter; all 32 lanes call.
__device__ __forceinline__ int warp_append(int* counter, bool want)
{
    const unsigned b = __ballot_sync(0xffffffffu, want);
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && b) base = atomicAdd(counter, __popc(b));
    base = __shfl_sync(0xffffffffu, base, 0);
    return base + __popc(b & ((1u << lane) - 1));
}

// Label of `key` in the voxel table (-1: absent), probed by the PW lanes of
// an aligned lane group together (warp-cooperative probing): each round the
// group loads PW consecutive slots of the probe sequence, and the first slot
// in probe order that holds the key or is empty decides.  All lanes of a
// group pass the same key and `active`; inactive groups return -1 at once.
// *probes: slots passed before the deciding one; *full: no empty slot found.
template <int PW>
__device__ __forceinline__ int probe_label(const VoxelTable& vt, unsigned long long key, bool active, int* probes,
                                           bool* full)
{
    *probes = 0;
    *full = false;
    if (!active) return -1;
    const int lane = threadIdx.x & 31, base = lane & ~(PW - 1), sub = lane - base;
    const unsigned gmask = (PW == 32 ? 0xffffffffu : ((1u << PW) - 1u)) << base;
    const unsigned long long h = mix64(key) & vt.mask;
    for (unsigned long long pr = 0; pr <= vt.mask; pr += PW) {
        const unsigned long long slot = (h + pr + sub) & vt.mask;
        const unsigned long long kk = vt.keys[slot];
        const unsigned hit = (__ballot_sync(gmask, kk == key || kk == EMPTY_KEY) & gmask) >> base;
        if (hit) {
            const int first = __ffs(hit) - 1;
            const bool found = __shfl_sync(gmask, kk == key, base + first);
            int lab = -1;
            if (found && sub == first) lab = vt.labels[slot];
            *probes = (int)pr + first;
            return found ? __shfl_sync(gmask, lab, base + first) : -1;
        }
    }
    *full = true;
    return -1;
}

// Every entry of every frame slot of the batch (block row = slot): its label
// in the map at the batch start (tag-0 item), or, when absent, its slot in
// the batch's absent-voxel hash, where the least (frame position, segment)
// containing it is kept.  PW lanes look each entry up together (PW = 1: one
// lane per entry); the group's first lane carries the entry afterwards.
template <int PW>
__global__ void __launch_bounds__(256) k_lookup(const FrameParams* fps, BatchScratch bs, const MapRefs* refs,
                                               AbsentHash ah)
{
    const int f = blockIdx.y;
    const FrameParams& fp = fps[f];
    const Scratch sc = bs.frame(f);
    const int ne = sc.ctr->n_entries;
    if (fp.M <= 0 || sc.ctr->err) return;  // a failed frame's items are never read
    const VoxelTable vt = refs[fp.map].vt;
    const unsigned long long gtag = (unsigned long long)(fp.map + 1) << 54;
    const int lane = threadIdx.x & 31;
    constexpr int PER = 32 / PW;  // entries of a warp per round
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    int maxp = 0;
    for (int i0 = warp * PER; i0 < ne; i0 += nwarps * PER) {  // whole warps iterate together
        const int i = i0 + lane / PW;
        const bool valid = i < ne;
        const bool lead = valid && (lane & (PW - 1)) == 0;
        const unsigned long long hk = valid ? sc.sent[i] : 0ull;
        const int m = (int)(hk >> 54);
        const unsigned long long key = hk & KEY54;
        int probes;
        bool full;
        const int lab = probe_label<PW>(vt, key, valid, &probes, &full);
        if (lead && full) set_err(sc.ctr, DISC_ERR_TABLE_FULL);
        maxp = max(maxp, probes);
        int at = -1;
        bool claimed = false;
        if (lead && !full && lab < 0) {
            const unsigned long long ak = gtag | key;
            unsigned long long t = mix64(ak) & ah.mask;
            for (unsigned long long pr = 0;; pr++) {
                const unsigned long long cur = ah.key[t];
                if (cur == ak) break;
                if (cur == 0ull) {
                    const unsigned long long prev = atomicCAS(&ah.key[t], 0ull, ak);
                    if (prev == 0ull) { claimed = true; break; }
                    if (prev == ak) break;
                }
                t = (t + 1) & ah.mask;
                if (pr > ah.mask) { set_err(sc.ctr, DISC_ERR_TABLE_FULL); t = ~0ull; break; }
            }
            if (t != ~0ull) {
                atomicMin(&ah.val[t], (fp.jpos << 9) | m);
                at = (int)t;
            }
        }
        add_item_warp(sc, ((unsigned long long)m << 33) | (unsigned)lab, lead && lab >= 0);
        const int li = warp_append(ah.n, claimed);
        if (claimed) ah.list[li] = at;
        const int ai = warp_append(&sc.ctr->n_absent, at >= 0);
        if (at >= 0) {
            sc.aent[ai] = i;
            sc.aslot[ai] = at;
        }
    }
    const int pm = __reduce_max_sync(0xffffffffu, maxp);
    if (lane == 0 && pm > 0) atomicMax(&sc.ctr->max_probe, pm);
}

// Every entry absent at the batch start, once the batch-wide hash holds each
// voxel's first (frame position j0, segment m0): j0 before this frame makes a
// tag-1 item (m, j0 << 9 | m0); j0 this frame makes a new voxel, counted for
// its owner m0 once (by the entry of m0 itself).
__global__ void __launch_bounds__(256) k_absent(const FrameParams* fps, BatchScratch bs, AbsentHash ah)
{
    __shared__ int s_new[MAX_MASKS];
    const int f = blockIdx.y;
    const FrameParams& fp = fps[f];
    const Scratch sc = bs.frame(f);
    const int na = sc.ctr->n_absent;
    if (fp.M <= 0 || sc.ctr->err || (int)(blockIdx.x * blockDim.x) >= na) return;  // uniform per block
    for (int m = threadIdx.x; m < fp.M; m += blockDim.x) s_new[m] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int a0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); a0 < na; a0 += gridDim.x * blockDim.x) {
        const int a = a0 + lane;
        const bool valid = a < na;
        int m = 0, pv = 0;
        if (valid) {
            m = (int)(sc.sent[sc.aent[a]] >> 54);
            pv = ah.val[sc.aslot[a]];
        }
        const int j0 = pv >> 9, m0 = pv & 511;
        add_item_warp(sc, ((unsigned long long)m << 33) | (1ull << 32) | (unsigned)pv, valid && j0 < fp.jpos);
        if (valid && j0 == fp.jpos && m0 == m) atomicAdd(&s_new[m - 1], 1);
    }
    __syncthreads();
    int tot = 0;
    for (int m = threadIdx.x; m < fp.M; m += blockDim.x)
        if (s_new[m]) {
            atomicAdd(&sc.newcnt[m], s_new[m]);
            tot += s_new[m];
        }
    tot = warp_sum(tot);
    if (lane == 0 && tot) atomicAdd(&sc.ctr->n_new, tot);
}

// Every slot's overlap items, once k_absent is done: the hash slots listed
// in plist become dense (key, count) arrays in claim order (ikey over the
// free aent | aslot, icnt over plist itself: each thread reads plist[i]
// before it writes icnt[i]), and the hash is emptied for the slot's next
// batch.  Items of a failed frame are emptied as well.
__global__ void __launch_bounds__(256) k_items(BatchScratch bs)
{
    const Scratch sc = bs.frame(blockIdx.y);
    const int n = sc.ctr->n_pre;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int t = sc.plist[i];
        const unsigned long long key = sc.pkey[t];
        const int cnt = sc.pcnt[t];
        sc.pkey[t] = EMPTY_KEY;
        sc.pcnt[t] = 0;
        sc.ikey[i] = key;
        sc.icnt[i] = cnt;
    }
}

// root of instance id x (parent chains may be longer than one step between
// the merges of a batch and its k_commit).  A parent is never above its
// child (a merge hooks an instance under the component's smallest id), so a
// chain ends within one step per merging frame of the batch; the step limit
// only keeps a damaged table from looping.
__device__ __forceinline__ int find_root(const int32_t* parent, int x)
{
    for (int it = 0; it < (1 << 16); it++) {
        const int p = parent[x];
        if (p == x) break;
        x = p;
    }
    return x;
}

// one thread reads a counter word another thread of the launch may have
// written by an atomic; every thread then takes the same branch
__device__ __forceinline__ int block_read(const int32_t* w)
{
    __shared__ int s_v;
    __syncthreads();
    if (threadIdx.x == 0) s_v = *(volatile const int32_t*)w;
    __syncthreads();
    const int v = s_v;
    __syncthreads();
    return v;
}

constexpr int ASSOC_THREADS = 512;
constexpr int APH = 2048;         // slots of the leader CTA's pair hash (shared memory)
constexpr int APH_MAX = 1536;     // pairs it takes (load <= 3/4)
constexpr int ASSOC_ROOTS = 256;  // instances with an accepted edge, in shared memory
constexpr int ASSOC_EDGES = 512;  // accepted edges, in shared memory
// A frame past one of these shared capacities runs steps (1)-(3) on the
// leader alone with the map's global pair hash and union region.  The small
// footprint lets the CTAs share SMs with the next batch's stateless kernels.
constexpr size_t ASSOC_SMEM = (size_t)APH * 16 + union_region_bytes(2 * APH, ASSOC_ROOTS, ASSOC_EDGES, true);
constexpr int ASSOC_CLUSTER_MAX = 8;
static_assert(ASSOC_EDGES >= 2 * ASSOC_ROOTS, "the fusion step overlays the edge arrays");

// ---- distributed shared memory of a thread-block cluster (inline PTX) ------------
// Addresses are 32-bit shared::cluster addresses: a CTA's own shared-memory
// offset mapped to the CTA of the given rank (mapa).
__device__ __forceinline__ unsigned dsm_map(const void* local, unsigned rank)
{
    unsigned out;
    const unsigned a = (unsigned)__cvta_generic_to_shared(local);
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(a), "r"(rank));
    return out;
}
__device__ __forceinline__ unsigned long long dsm_cas64(unsigned a, unsigned long long cmp, unsigned long long v)
{
    unsigned long long old;
    asm volatile("atom.shared::cluster.cas.b64 %0, [%1], %2, %3;" : "=l"(old) : "r"(a), "l"(cmp), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ int dsm_add(unsigned a, int v)
{
    int old;
    asm volatile("atom.shared::cluster.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(a), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void dsm_red_add(unsigned a, int v)
{
    asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long dsm_ld64(unsigned a)
{
    unsigned long long v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ int dsm_ld32(unsigned a)
{
    int v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void dsm_st32(unsigned a, int v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void dsm_st64(unsigned a, unsigned long long v)
{
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size()
{
    unsigned n;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
    return n;
}
// every thread of every CTA of the cluster; shared-memory and global writes
// before it are visible to the cluster after it (release / acquire)
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// the two halves of cluster_sync: between them a thread may read what no
// other thread of the cluster writes in this phase
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }

// A cluster of C CTAs per map of the batch (C = cluster size, 1 to 8)
// walks the map's frames in order.  The leader CTA (rank 0) holds the
// frame's pair hash, scored-pair list, edge list and union state in its
// shared memory; the other CTAs reach them through distributed shared
// memory.  Per frame:
//   (1) every CTA resolves a share of the frame's items to (segment, root)
//       pairs and counts them in the leader's pair hash;
//   (2) every thread of the cluster checks the overlap gate of one pair and
//       appends a passing pair to the scored list; then every warp takes the
//       cosine gate of one scored pair (so no warp scores several while
//       others idle); accepted edges go to the leader's edge list;
//   (3) the leader alone: union, new ids, merges and fusion winners; then it
//       stages the frame's status and copy count and empties its pair hash;
//   (4) every warp a share of the embedding copies; the leader the voxel
//       counts of the frame's new voxels;
// with a cluster barrier after (1), after each half of (2) and after (3).
// Step (4) needs no barrier before the next frame's step (1): that step
// touches only the leader's emptied hash, and the next barrier orders the
// copies before the next gates read the embeddings.  The status and copy
// count alternate between two words by frame parity, so the leader may
// stage the next frame's while a slower CTA still reads this frame's.  A
// frame with more pairs than the leader's hash takes (APH_MAX), or more
// edges or edge roots than its union region holds, runs steps (1)-(3) on the
// leader alone with the map's global pair hash.  Every branch that skips a
// cluster barrier is taken by the whole cluster (its condition is read from
// global memory written before the launch, or from the leader after a
// barrier), so every CTA passes the same barriers.
__global__ void __launch_bounds__(ASSOC_THREADS, 1) k_associate(const FrameParams* fps, BatchScratch bs,
                                                                SerialStep st)
{
    extern __shared__ __align__(16) unsigned char union_smem[];
    __shared__ int s_np, s_ovf, s_ne, s_nsc, s_merged;
    __shared__ int s_err[2], s_nc[2];  // by frame parity
    const unsigned rank = cluster_rank(), C = cluster_size();
    const bool leader = rank == 0;
    const int g = blockIdx.x / C;
    const int tid = threadIdx.x, lane = tid & 31, NT = blockDim.x;
    // the map's table pointers, in shared memory: read there, they are never
    // reloaded from global memory after the kernel's own global stores
    __shared__ MapRefs s_refs;
    static_assert(sizeof(MapRefs) % 8 == 0, "copied in 8-byte words");
    for (int i = tid; i < (int)(sizeof(MapRefs) / 8); i += NT)
        ((unsigned long long*)&s_refs)[i] = ((const unsigned long long*)&st.refs[g])[i];
    __syncthreads();
    const MapRefs& R = s_refs;
    const int ct = (int)rank * NT + tid, CT = (int)C * NT;               // thread within the cluster
    const int cw = (int)rank * (NT >> 5) + (tid >> 5), CW = (int)C * (NT >> 5);  // warp within the cluster
    // the leader's step (1)-(3) state, laid out as in its union_smem:
    // pair hash, then the union's region (root hash of 2 * APH slots,
    // per-root arrays, edges); the scored pairs (segment, instance) sit over
    // the root hash, which the union fills only after the gates
    unsigned long long* pk = (unsigned long long*)union_smem;  // [APH] (segment + 1) << 32 | root
    int* pc = (int*)(pk + APH);                                 // [APH] voxels of the pair
    int* pl = pc + APH;                                         // [APH] used slots
    unsigned char* ureg = union_smem + (size_t)APH * 16;
    int2* sp = (int2*)ureg;                                     // [APH_MAX] scored pairs
    const UnionRegion U(ureg, 2 * APH, ASSOC_ROOTS, ASSOC_EDGES, true);
    static_assert((size_t)APH_MAX * 8 <= (size_t)(2 * APH) * 8, "scored pairs fit over the root hash");
    const unsigned r_pk = dsm_map(pk, 0), r_pc = dsm_map(pc, 0), r_pl = dsm_map(pl, 0), r_sp = dsm_map(sp, 0);
    const unsigned r_em = dsm_map(U.em, 0), r_ek = dsm_map(U.ek, 0), r_ec = dsm_map(U.ec, 0);
    const unsigned r_eq = dsm_map(U.eq, 0), r_eo = dsm_map(U.eo, 0);
    const unsigned r_np = dsm_map(&s_np, 0), r_ovf = dsm_map(&s_ovf, 0), r_ne = dsm_map(&s_ne, 0);
    const unsigned r_nsc = dsm_map(&s_nsc, 0), r_err = dsm_map(&s_err[0], 0), r_nc = dsm_map(&s_nc[0], 0);
    if (leader) {
        for (int i = tid; i < APH; i += NT) {
            pk[i] = EMPTY_KEY;
            pc[i] = 0;
        }
        if (tid == 0) {
            *R.ss.edge_n = 0;
            *R.ss.copy_n = 0;
            s_merged = 0;
            s_np = s_ovf = s_ne = s_nsc = 0;
            s_err[0] = s_err[1] = 0;
            s_nc[0] = s_nc[1] = 0;
        }
    }
    cluster_sync();
    for (int j = 0; j < st.J; j++) {
        const int slot = st.slot_of[g * st.J + j];  // the same for the whole cluster
        if (slot < 0) break;
        const int par = j & 1;
        const FrameParams& fp = fps[slot];
        const Scratch sc = bs.frame(slot);
        // blocked: the frame's own error (set before the launch), or its
        // predecessor's status (staged by the leader before the last barrier)
        const int prev = j > 0 ? dsm_ld32(r_err + 4u * (par ^ 1))
                               : (st.prev_hist[g] >= 0 ? st.hist[st.prev_hist[g]].err : 0);
        const int own = *(volatile const int32_t*)&sc.ctr->err;
        const bool blocked = own || prev;
        if (leader && tid == 0 && !own && prev) set_err(sc.ctr, prev);
        bool global_pairs = false;
        // the leader's per-segment union inputs; up.ok: the union completed
        // (and added the frame's new voxels to the counts)
        UnionPre up{};
        if (!blocked) {
            const int npre = sc.ctr->n_pre;
            // (1) overlap pairs: each item's label resolved to its root now
            //     (four items per thread in flight)
            for (int i0 = ct; i0 < npre; i0 += 4 * CT) {
                unsigned long long key[4];
                int cnt[4], lab[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int i = i0 + u * CT;
                    key[u] = i < npre ? sc.ikey[i] : EMPTY_KEY;
                    cnt[u] = i < npre ? sc.icnt[i] : 0;
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const unsigned x = (unsigned)key[u];
                    lab[u] = -1;
                    if (key[u] != EMPTY_KEY)
                        lab[u] = ((key[u] >> 32) & 1ull)
                                     ? bs.frame(st.slot_of[g * st.J + (int)(x >> 9)]).segrep[(x & 511u) - 1]
                                     : (int)x;
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    if (lab[u] < 0) continue;
                    const unsigned long long okey = ((key[u] >> 33) << 32) | (unsigned)find_root(R.inst.parent, lab[u]);
                    unsigned h = (unsigned)(mix64(okey) & (APH - 1));
                    for (int pr = 0;; pr++) {  // claim or find in one round trip per slot
                        const unsigned long long prv = dsm_cas64(r_pk + 8u * h, EMPTY_KEY, okey);
                        if (prv == EMPTY_KEY) {
                            const int at = dsm_add(r_np, 1);
                            if (at < APH_MAX) dsm_st32(r_pl + 4u * at, (int)h);
                            else dsm_st32(r_ovf, 1);
                            break;
                        }
                        if (prv == okey) break;
                        h = (h + 1) & (APH - 1);
                        if (pr >= APH) {
                            dsm_st32(r_ovf, 1);
                            break;
                        }
                    }
                    dsm_red_add(r_pc + 4u * h, cnt[u]);
                }
            }
            cluster_sync();
            global_pairs = dsm_ld32(r_ovf) != 0;  // the whole cluster
            if (!global_pairs) {
                const int np = dsm_ld32(r_np);
                // (2a) overlap gate of pair i by thread i of the cluster:
                //      |V_m & V_k| / min(|V_m|, |V_k|) >= ov_num / ov_den;
                //      passing pairs to the scored list (one slot claim per warp)
                for (int w0 = ct & ~31; w0 < np; w0 += CT) {  // whole warps iterate together
                    const int i = w0 + lane;
                    int m = 0, k = 0;
                    bool pass = false;
                    if (i < np) {
                        const unsigned h = (unsigned)dsm_ld32(r_pl + 4u * i);
                        const unsigned long long okey = dsm_ld64(r_pk + 8u * h);
                        const long long ov = dsm_ld32(r_pc + 4u * h);
                        m = (int)(okey >> 32) - 1;
                        k = (int)(okey & 0xffffffffu);
                        const long long denom = min((long long)sc.nvox[m], R.inst.count[k]);
                        pass = ov * (long long)fp.ov_den >= (long long)fp.ov_num * denom;
                    }
                    const unsigned b = __ballot_sync(0xffffffffu, pass);
                    int base = 0;
                    if (lane == 0 && b) base = dsm_add(r_nsc, __popc(b));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (pass) {
                        const unsigned at = (unsigned)(base + __popc(b & ((1u << lane) - 1)));
                        dsm_st32(r_sp + 8u * at, m);
                        dsm_st32(r_sp + 8u * at + 4u, k);
                    }
                }
                cluster_sync();
                const int nsc = dsm_ld32(r_nsc);
                if (leader && tid == 0) {
                    sc.ctr->n_pairs = np;
                    sc.ctr->n_scored = nsc;
                }
                // (2b) cosine gate of scored pair s by warp s of the cluster
                const GateFeatures gf = gate_features(fp, sc, st.view.frame(slot), R.inst);
                int border = 0;
                for (int q = cw; q < nsc; q += CW) {
                    const int mm = dsm_ld32(r_sp + 8u * q), kk = dsm_ld32(r_sp + 8u * q + 4u);
                    // the instance's values the union needs, read beside the gate
                    const long long ck = lane == 0 ? R.inst.count[kk] : 0;
                    const float qk = lane == 0 ? R.inst.Q[kk] : 0.0f;
                    const int ok = lane == 0 ? R.inst.n_obs[kk] : 0;
                    if (warp_cosine_gate(fp, gf, R.inst, mm, kk, &border) && lane == 0) {
                        const int e = dsm_add(r_ne, 1);
                        if (e < ASSOC_EDGES) {
                            dsm_st32(r_em + 4u * e, mm);
                            dsm_st32(r_ek + 4u * e, kk);
                            dsm_st64(r_ec + 8u * e, (unsigned long long)ck);
                            dsm_st32(r_eq + 4u * e, __float_as_int(qk));
                            dsm_st32(r_eo + 4u * e, ok);
                        }  // more edges than the shared list holds: the global path below
                    }
                }
                if (lane == 0 && border) atomicAdd(&sc.ctr->borderline, border);
                // the leader reads its segments' values for the union while
                // the cluster arrives (nothing in the cluster writes them)
                cluster_arrive();
                if (leader) {
                    if (tid < fp.M) {
                        up.nv = sc.nvox[tid];
                        up.q = sc.S[5 * tid + 4];
                        up.nnew = sc.newcnt[tid];
                    }
                    up.next = *(volatile const int*)R.next_id;
                }
                cluster_wait();
                // (3) union, new ids, merges, fusion winners: the leader, in
                //     its shared memory unless a shared capacity is exceeded
                if (leader) {
                    bool done = s_ne <= ASSOC_EDGES;
                    if (done && !block_read(&sc.ctr->err)) {
                        done = union_frame(fp, sc, R.ss, R.inst, R.next_id, ureg, 2 * APH, ASSOC_ROOTS, ASSOC_EDGES,
                                           true, np, s_ne, true, [&](int i) { return (unsigned)(pk[pl[i]] & 0xffffffffu); },
                                           &up);
                    }
                    if (!done && tid == 0) {  // steps (1)-(3) again on global memory
                        sc.ctr->n_pairs = 0;
                        sc.ctr->n_scored = 0;
                        sc.ctr->borderline = 0;
                    }
                    global_pairs = !done;  // uniform in the leader
                }
            }
            if (leader && global_pairs) {
                // more pairs, edges or edge roots than the leader's shared
                // memory holds: the leader alone, with the map's global pair
                // hash and union region
                __syncthreads();
                for (int i = tid; i < npre; i += NT) {
                    const unsigned long long key = sc.ikey[i];
                    const unsigned x = (unsigned)key;
                    const int lab = ((key >> 32) & 1ull)
                                        ? bs.frame(st.slot_of[g * st.J + (int)(x >> 9)]).segrep[(x & 511u) - 1]
                                        : (int)x;
                    if (lab >= 0)
                        add_pair(sc, R.ss, ((key >> 33) << 32) | (unsigned)find_root(R.inst.parent, lab), sc.icnt[i]);
                }
                if (!block_read(&sc.ctr->err))
                    phase_score(fp, sc, st.view.frame(slot), R.ss, R.inst, tid >> 5, NT >> 5);
                if (!block_read(&sc.ctr->err)) phase_union(fp, sc, R.ss, R.inst, R.next_id, R.ss.ureg);
                // empty the global pair hash
                __syncthreads();
                const int np = *(volatile int32_t*)&sc.ctr->n_pairs;
                for (int i = tid; i < np; i += NT) {
                    const int t = R.ss.olist[i];
                    R.ss.okeys[t] = EMPTY_KEY;
                    R.ss.ocnt[t] = 0;
                }
            }
        }
        // the leader closes the frame: its status and copy count for step (4)
        // and the next frame, its pair hash emptied for the next frame
        if (leader) {
            __syncthreads();
            const int err = up.ok ? 0 : *(volatile int32_t*)&sc.ctr->err;
            const int nc = up.ok ? up.ncopy : err ? 0 : *(volatile int32_t*)R.ss.copy_n;
            for (int i = tid; i < APH; i += NT) {
                pk[i] = EMPTY_KEY;
                pc[i] = 0;
            }
            if (tid == 0) {
                s_err[par] = err;
                s_nc[par] = nc;
                s_np = s_ovf = s_ne = s_nsc = 0;
            }
        }
        cluster_sync();
        // (4) the winners' embeddings (every warp of the cluster) and the
        //     new voxels' counts (the leader)
        if (!dsm_ld32(r_err + 4u * par)) {
            const int D = fp.D;
            const int nc = dsm_ld32(r_nc + 4u * par);
            // from the cluster's last warp down: the first warps take the
            // next frame's items, so the two run side by side
            for (int c = CW - 1 - cw; c < nc; c += CW) {
                const int src = R.ss.copy_src[c], dst = R.ss.copy_dst[c];
                const Instances& inst = R.inst;
                const float* from = src >= 0 ? inst.E + (size_t)src * D : sc.Ecan + (size_t)(-src - 1) * D;
                if (inst.A) {
                    const Scratch va = st.view.frame(slot);
                    const int Da = inst.Da;
                    const float* fa = src >= 0 ? inst.A + (size_t)src * Da : va.Ecan + (size_t)(-src - 1) * Da;
                    copy_row(from, inst.E + (size_t)dst * D, nullptr, D, lane);
                    copy_row(fa, inst.A + (size_t)dst * Da, inst.Eb ? inst.Eb + (size_t)dst * Da : nullptr, Da, lane);
                    if (inst.E8) e4m3_copy_row(fa, Da, inst.E8 + (size_t)dst * Da, inst.Er + dst);
                } else {
                    copy_row(from, inst.E + (size_t)dst * D, inst.Eb ? inst.Eb + (size_t)dst * D : nullptr, D, lane);
                    if (inst.E8) e4m3_copy_row(from, D, inst.E8 + (size_t)dst * D, inst.Er + dst);
                }
            }
            if (leader) {
                for (int m = tid; m < fp.M && !up.ok; m += NT) {
                    const int n = sc.newcnt[m], rep = sc.segrep[m];
                    if (n && rep >= 0) atomicAdd((unsigned long long*)&R.inst.count[rep], (unsigned long long)n);
                }
                if (tid == 0 && (up.ok ? up.merges : sc.ctr->merges) > 0) s_merged = 1;
            }
        }
        if (leader && tid == 0) {
            *R.ss.edge_n = 0;
            *R.ss.copy_n = 0;
        }
    }
    // no CTA leaves while another may still reach its shared memory
    cluster_sync();
    if (leader && tid == 0) st.merged[g] = s_merged;
}

// After the batch's frames: every voxel of the absent-voxel hash whose first
// frame succeeded goes into its map with the instance that frame's lowest
// segment joined; the hash is emptied on the way.  Then the parent table of
// every map whose frames merged is flattened (each id to its root).
__global__ void k_commit(BatchScratch bs, SerialStep st, AbsentHash ah, int G)
{
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int n = *ah.n;
    for (int i0 = gtid & ~31; i0 < n; i0 += gsz) {
        const int i = i0 + lane;
        int g = -1, lab = -1;
        unsigned long long key = 0;
        if (i < n) {
            const int t = ah.list[i];
            const unsigned long long ak = ah.key[t];
            const int pv = ah.val[t];
            ah.key[t] = 0ull;
            ah.val[t] = INT_MAX;
            g = (int)(ak >> 54) - 1;
            key = ak & KEY54;
            const int slot = st.slot_of[g * st.J + (pv >> 9)];
            const Scratch sc = bs.frame(slot);
            if (sc.ctr->err == 0) lab = sc.segrep[(pv & 511) - 1];
        }
        const bool ins = lab >= 0;
        if (ins) {
            const VoxelTable vt = st.refs[g].vt;
            unsigned long long h = mix64(key) & vt.mask;
            for (unsigned long long pr = 0;; pr++) {
                const unsigned long long prev = atomicCAS(&vt.keys[h], EMPTY_KEY, key);
                if (prev == EMPTY_KEY) {
                    vt.labels[h] = lab;
                    break;
                }
                h = (h + 1) & vt.mask;
                if (pr > vt.mask) break;  // not reached: the batch's room was checked before it ran
            }
        }
        // one count update per map of the warp
        const unsigned act = __ballot_sync(0xffffffffu, ins);
        if (ins) {
            const unsigned grp = __match_any_sync(act, g);
            if (lane == __ffs(grp) - 1) atomicAdd(st.refs[g].vt.used, (unsigned long long)__popc(grp));
        }
    }
    for (int g = 0; g < G; g++) {
        if (!st.merged[g]) continue;
        const Instances inst = st.refs[g].inst;
        const int nid = *st.refs[g].next_id;
        for (int i = gtid; i < nid; i += gsz) inst.parent[i] = find_root(inst.parent, i);
    }
}

// ---- host launcher ----------------------------------------------------------------
// E4M3 scoring copies of instances [0, n) from their scoring master (one
// warp per instance), as the apply phase writes them
__global__ void k_e4m3_copies(Instances inst, int n, int D)
{
    const float* Sm = scoring_master(inst);
    const int Ds = scoring_dim(inst, D);
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += (gridDim.x * blockDim.x) >> 5)
        e4m3_copy_row(Sm + (size_t)k * Ds, Ds, inst.E8 + (size_t)k * Ds, inst.Er + k);
}

int launch_e4m3_copies(const Instances& inst, int n, int D, cudaStream_t st)
{
    if (n <= 0 || !inst.E8) return 0;
    k_e4m3_copies<<<std::min((n + 7) / 8, 1216), 256, 0, st>>>(inst, n, D);
    return 1;
}

// Room check between a batch's two parts: per map of the batch, its voxel
// count (after every earlier batch) and the unique (segment, voxel) pairs of
// its frames in this batch, an upper bound of the voxels the batch inserts.
__global__ void k_room(const MapRefs* refs, int G, const int* slot_of, int J, BatchScratch bs,
                       unsigned long long* out)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        unsigned long long inc = 0;
        for (int j = 0; j < J; j++) {
            const int slot = slot_of[g * J + j];
            if (slot >= 0) inc += (unsigned long long)max(bs.frame(slot).ctr->n_entries, 0);
        }
        out[2 * g] = *refs[g].vt.used;
        out[2 * g + 1] = inc;
    }
}

int launch_room(const MapRefs* refs, int G, const int* slot_of, int J, const BatchScratch& bs, unsigned long long* out,
                cudaStream_t st)
{
    k_room<<<(G + 127) / 128, 128, 0, st>>>(refs, G, slot_of, J, bs, out);
    return 1;
}

int launch_serial_begin(const MapRefs* refs, int G, cudaStream_t st)
{
    k_serial_begin<<<(G + 127) / 128, 128, 0, st>>>(refs, G);
    return 1;
}

// Blocks per map: the whole GPU for a single map, fewer per map as the maps
// of a batch multiply (they run side by side).
static int per_map(int full, int G, int least)
{
    return std::max(least, (full + G - 1) / G);
}

int launch_serial_step(const FrameParams* fps, const BatchScratch& bs, const SerialStep& st, int G, int phase,
                       cudaStream_t st_)
{
    const int q = st.cta_scale > 0 ? st.cta_scale : 4;  // quarters of the default CTA counts
    switch (phase) {
        case 0:
            k_overlap<<<dim3(per_map(76 * 2 * q / 2, G, 8), G), SER_THREADS, OV_SMEM, st_>>>(fps, bs, st);
            return 1;
        case 1:
            k_score<<<dim3(per_map(38 * q, G, 4), G), 256, 0, st_>>>(fps, bs, st);
            return 1;
        case 2:
            k_union<<<dim3(1, G), UNION_THREADS, UNION_SMEM, st_>>>(fps, bs, st);
            return 1;
        default:
            k_apply<<<dim3(per_map(76 * q, G, 8), G), 256, 0, st_>>>(fps, bs, st);
            return 1;
    }
}

int launch_lookup(const FrameParams* fps, const BatchScratch& bs, const MapRefs* refs, const AbsentHash& ah, int S,
                  int probe_width, cudaStream_t st)
{
    const dim3 grid(152, S);
    switch (probe_width) {
        case 2: k_lookup<2><<<grid, 256, 0, st>>>(fps, bs, refs, ah); break;
        case 4: k_lookup<4><<<grid, 256, 0, st>>>(fps, bs, refs, ah); break;
        case 8: k_lookup<8><<<grid, 256, 0, st>>>(fps, bs, refs, ah); break;
        default: k_lookup<1><<<grid, 256, 0, st>>>(fps, bs, refs, ah); break;
    }
    k_absent<<<dim3(38, S), 256, 0, st>>>(fps, bs, ah);
    k_items<<<dim3(16, S), 256, 0, st>>>(bs);
    return 3;
}

// CTAs per map: a cluster of up to 8 when the maps leave SMs free (152 SMs,
// one CTA each); checked once against what the device can co-schedule.
static int g_assoc_max_cluster = -1;  // set once by set_serial_kernel_attrs

static void probe_assoc_cluster()
{
    if (g_assoc_max_cluster < 0) {
        int& max_c = g_assoc_max_cluster;
        max_c = 1;
        for (int c = ASSOC_CLUSTER_MAX; c > 1; c >>= 1) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = c;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(c);
            cfg.blockDim = dim3(ASSOC_THREADS);
            cfg.dynamicSmemBytes = ASSOC_SMEM;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, k_associate, &cfg) == cudaSuccess && n > 0) {
                max_c = c;
                break;
            }
            cudaGetLastError();
        }
    }
}

static int assoc_cluster(int G, int want)
{
    int c = 1;
    if (want > 0) {
        while (c * 2 <= want && c * 2 <= g_assoc_max_cluster) c *= 2;
        return c;
    }
    while (c * 2 <= g_assoc_max_cluster && (c * 2) * G <= 152) c *= 2;
    return c;
}

size_t union_region_bytes_full() { return UNION_SMEM; }

int launch_associate(const FrameParams* fps, const BatchScratch& bs, const SerialStep& st, int G, int cluster,
                     cudaStream_t s)
{
    const int c = assoc_cluster(G, cluster);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(G * c);
    cfg.blockDim = dim3(ASSOC_THREADS);
    cfg.dynamicSmemBytes = ASSOC_SMEM;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_associate, fps, bs, st);
    return 1;
}

int launch_commit(const BatchScratch& bs, const SerialStep& st, const AbsentHash& ah, int G, cudaStream_t s)
{
    k_commit<<<152 * 2, 512, 0, s>>>(bs, st, ah, G);
    return 1;
}

cudaError_t set_serial_kernel_attrs()
{
    cudaError_t e = cudaFuncSetAttribute(k_union, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)UNION_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_associate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ASSOC_SMEM);
    if (e == cudaSuccess) probe_assoc_cluster();
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_overlap, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OV_SMEM);
    return e;
}

}  // namespace disc
