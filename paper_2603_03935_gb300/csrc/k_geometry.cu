// Geometry kernels of the integration step, batched over the frames of a batch
// (they only read the map):
//   Sec. III-A  masked depth -> world points -> voxel keys and pixel normals;
//               per-segment voxel sets V_m in the frame slot's hash
//   Eq. 3       per voxel max(0, -r_v . n_v), summed exactly per segment
//   Sec. III-B  label of every voxel in the map as it stood at the start of
//               the batch (voxels absent then are re-probed by the serial
//               overlap kernel, which sees the inserts of earlier frames)
//   Eq. 2       Q = S_size * S_angle * S_sem * S_dist per segment
#include <algorithm>
#include <climits>

#include "disc_common.cuh"
#include "kernels.h"

namespace disc {

__device__ __forceinline__ void set_err(FrameCounters* c, int code) { atomicCAS(&c->err, 0, code); }

// ---- slot clearing: the hashes and accumulators a frame slot used last time --
__global__ void k_slot_clear(BatchScratch bs, int D, int MM)
{
    const Scratch sc = bs.frame(blockIdx.y);
    const int ne = sc.ctr->n_entries;
    const int nc = sc.dkey ? sc.ctr->n_cells : 0;
    const int n = max(max(ne, nc), max(D, MM));
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < ne) sc.sslot[sc.slist[i]] = SegSlot{0ull, {0, 0, 0}};
        if (i < nc) {
            sc.dkey[sc.dlist[i]] = 0ull;
            sc.dcnt[sc.dlist[i]] = 0;
        }
        if (i < D) sc.sumF[i] = 0;
        if (i < MM) {
            sc.npix[i] = 0;
            sc.ang[i] = 0;
            sc.nvox[i] = 0;
            sc.segrep[i] = -1;
            if (sc.newcnt) sc.newcnt[i] = 0;
        }
    }
}

// counters and scalar sums of every slot (after k_slot_clear has read them)
__global__ void k_slot_reset(BatchScratch bs, int B)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const Scratch sc = bs.frame(b);
    *sc.gg = 0;
    *sc.nsum = 0;
    FrameCounters z = {};
    *sc.ctr = z;
}

// ---- back-projection + per-segment voxel dedupe (one thread per pixel) ----------
// A block covers a 32 x 16 pixel tile.  The tile and a one-pixel halo are
// loaded once into shared memory together with each position's world point,
// so neighbours' points (for the pixel normal) are read, not recomputed.
// The tile's pixels then meet in a shared hash keyed by (mask, voxel) that
// sums their normals exactly; only the tile's distinct keys update the frame
// slot's global hash.
constexpr int BP_TX = 32, BP_TY = 16, BP_THREADS = BP_TX * BP_TY;
constexpr int BP_HX = BP_TX + 2, BP_HY = BP_TY + 2, BP_HALO = BP_HX * BP_HY;
constexpr int BP_SLOTS = 2 * BP_THREADS;

struct __align__(16) TilePoint {
    float p[3];
    int lab;   // mask label if the pixel has valid depth (and is inside the image), else 0
};

__global__ void __launch_bounds__(BP_THREADS) k_backproject(const FrameParams* fps, BatchScratch bs, int f0)
{
    __shared__ TilePoint tp[BP_HALO];
    __shared__ unsigned long long tkey[BP_SLOTS];
    __shared__ int tn[6][BP_SLOTS];  // per component: sum of (v >> 16) and of (v & 0xffff)
    __shared__ unsigned short tlist[BP_THREADS];  // claimed tile slots
    __shared__ int tcount[3];        // valid pixels, dropped pixels, listed slots
    const FrameParams& fp = fps[f0 + blockIdx.z];
    const Scratch sc = bs.frame(f0 + blockIdx.z);
    if (fp.M <= 0) return;  // uniform per block
    const int tid = threadIdx.y * BP_TX + threadIdx.x;
    const int u0 = blockIdx.x * BP_TX - 1, v0 = blockIdx.y * BP_TY - 1;  // halo origin
    const bool ok_frame = !sc.ctr->err;
    // tile + halo: label (0 unless the depth is valid) and world point
    for (int i = tid; i < BP_HALO; i += BP_THREADS) {
        const int hu = u0 + i % BP_HX, hv = v0 + i / BP_HX;
        TilePoint t;
        t.lab = 0;
        t.p[0] = t.p[1] = t.p[2] = 0.0f;
        if (ok_frame && hu >= 0 && hv >= 0 && hu < fp.W && hv < fp.H) {
            const size_t idx = (size_t)hv * fp.W + hu;
            const int lab = fp.labels[idx];
            const float z = fp.depth[idx];
            // a DBSCAN noise pixel counts as invalid depth
            if (lab >= 1 && lab <= fp.M && z >= fp.z_min && z <= fp.z_max &&
                !(fp.db_min_pts > 0 && (sc.dflag[idx] & 2))) {
                t.lab = lab;
                world_point(fp, hu, hv, z, t.p);
            }
        }
        tp[i] = t;
    }
    for (int i = tid; i < BP_SLOTS; i += BP_THREADS) {
        tkey[i] = 0ull;
#pragma unroll
        for (int r = 0; r < 6; r++) tn[r][i] = 0;
    }
    if (tid < 3) tcount[tid] = 0;
    __syncthreads();
    const int hx = threadIdx.x + 1, hy = threadIdx.y + 1;  // own position in the halo tile
    const TilePoint me = tp[hy * BP_HX + hx];
    const int lab = me.lab;
    const bool active = lab > 0 && sc.npix[lab - 1] >= fp.min_px;
    unsigned long long key = 0;
    bool keyed = false;
    if (active) keyed = voxel_key(me.p[0], me.p[1], me.p[2], fp.inv_voxel, &key);
    const int lane = threadIdx.x & 31;
    const unsigned nvalid = __popc(__ballot_sync(0xffffffffu, keyed));
    const unsigned ndrop = __popc(__ballot_sync(0xffffffffu, active && !keyed));
    if (lane == 0) {
        if (nvalid) atomicAdd(&tcount[0], (int)nvalid);
        if (ndrop) atomicAdd(&tcount[1], (int)ndrop);
    }
    // pixel normal (zero when it has none)
    long long nfix[3] = {0, 0, 0};
    if (keyed) {
        // image-space tangents: forward differences, backward at the mask's
        // edge; a neighbour counts if it has valid depth and the same label
        const TilePoint& R = tp[hy * BP_HX + hx + 1];
        const TilePoint& L = tp[hy * BP_HX + hx - 1];
        const TilePoint& Dn = tp[(hy + 1) * BP_HX + hx];
        const TilePoint& Up = tp[(hy - 1) * BP_HX + hx];
        const float *pa = nullptr, *pb = nullptr, *qa = nullptr, *qb = nullptr;
        if (R.lab == lab) { pa = R.p; pb = me.p; }
        else if (L.lab == lab) { pa = me.p; pb = L.p; }
        if (Dn.lab == lab) { qa = Dn.p; qb = me.p; }
        else if (Up.lab == lab) { qa = me.p; qb = Up.p; }
        if (pa && qa) {
            float e1[3], e2[3], n[3];
#pragma unroll
            for (int r = 0; r < 3; r++) {
                e1[r] = __fsub_rn(pa[r], pb[r]);
                e2[r] = __fsub_rn(qa[r], qb[r]);
            }
            n[0] = __fsub_rn(__fmul_rn(e2[1], e1[2]), __fmul_rn(e2[2], e1[1]));
            n[1] = __fsub_rn(__fmul_rn(e2[2], e1[0]), __fmul_rn(e2[0], e1[2]));
            n[2] = __fsub_rn(__fmul_rn(e2[0], e1[1]), __fmul_rn(e2[1], e1[0]));
            float l2 = __fadd_rn(__fadd_rn(__fmul_rn(n[0], n[0]), __fmul_rn(n[1], n[1])), __fmul_rn(n[2], n[2]));
            if (l2 > 0.0f) {
                const float il = __frcp_rn(__fsqrt_rn(l2));
#pragma unroll
                for (int r = 0; r < 3; r++) n[r] = __fmul_rn(n[r], il);
                // orient toward the camera
                float vd = __fadd_rn(__fadd_rn(__fmul_rn(__fsub_rn(me.p[0], fp.t[0]), n[0]),
                                               __fmul_rn(__fsub_rn(me.p[1], fp.t[1]), n[1])),
                                     __fmul_rn(__fsub_rn(me.p[2], fp.t[2]), n[2]));
                if (vd > 0.0f) {
#pragma unroll
                    for (int r = 0; r < 3; r++) n[r] = -n[r];
                }
#pragma unroll
                for (int r = 0; r < 3; r++) nfix[r] = fix32f(n[r], S_VEC);
            }
        }
    }
    // Every keyed pixel adds its normal to its (mask, voxel) slot of the
    // tile's shared hash: each 2^-32 fixed-point component v (|v| <= 2^32)
    // splits exactly into v = (v >> 16) * 2^16 + (v & 0xffff), whose parts
    // add in 32-bit integers for up to a whole tile.  (Summing a warp's equal
    // keys first with a warp match and reductions measured 27 against 16 us
    // per frame: those warp instructions cost more than the shared-memory
    // atomics they save.)  The pixel that claims a slot lists it.
    if (keyed) {
        const unsigned long long hk = ((unsigned long long)lab << 54) | key;
        // tile-level dedupe: at most BP_THREADS distinct keys in BP_SLOTS slots
        unsigned t = (unsigned)(mix64(hk) & (BP_SLOTS - 1));
        while (true) {
            const unsigned long long cur = tkey[t];
            if (cur == hk) break;
            if (cur == 0ull) {
                const unsigned long long prev = atomicCAS(&tkey[t], 0ull, hk);
                if (prev == 0ull) {
                    tlist[atomicAdd(&tcount[2], 1)] = (unsigned short)t;
                    break;
                }
                if (prev == hk) break;
            }
            t = (t + 1) & (BP_SLOTS - 1);
        }
#pragma unroll
        for (int r = 0; r < 3; r++) {
            const unsigned hi = (unsigned)(int)(nfix[r] >> 16), lo = (unsigned)(nfix[r] & 0xffff);
            if (hi) atomicAdd((unsigned*)&tn[2 * r][t], hi);
            if (lo) atomicAdd((unsigned*)&tn[2 * r + 1][t], lo);
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (tcount[0]) atomicAdd(&sc.ctr->valid_pixels, tcount[0]);
        if (tcount[1]) atomicAdd(&sc.ctr->dropped_pixels, tcount[1]);
    }
    // the tile's distinct keys update the frame slot's hash, one lane per key
    // (whole warps iterate together); each warp appends the keys it claimed
    // first to the entry list with one reservation
    const int nkeys = tcount[2];
    const int warp = tid >> 5;
    int probes = 0;
    for (int i0 = warp * 32; i0 < nkeys; i0 += BP_THREADS) {
        const int i = i0 + lane;
        unsigned long long hk2 = 0ull;
        long long s = -1;
        bool claimed = false;
        if (i < nkeys) {
            const int t = tlist[i];
            hk2 = tkey[t];
            unsigned long long h = mix64(hk2) & sc.smask;
            while (true) {
                const unsigned long long cur = sc.sslot[h].key;
                if (cur == hk2) break;
                if (cur == 0ull) {
                    const unsigned long long prev = atomicCAS(&sc.sslot[h].key, 0ull, hk2);
                    if (prev == 0ull) {
                        claimed = true;
                        break;
                    }
                    if (prev == hk2) break;
                }
                h = (h + 1) & sc.smask;
                if (++probes > (int)sc.smask) {
                    set_err(sc.ctr, DISC_ERR_TABLE_FULL);
                    h = ~0ull;
                    break;
                }
            }
            if (h != ~0ull) {
                s = (long long)h;
                SegSlot& slot = sc.sslot[h];
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    const long long v = (long long)tn[2 * r][t] * 65536 + (long long)(unsigned)tn[2 * r + 1][t];
                    if (v) atomicAdd((unsigned long long*)&slot.n[r], (unsigned long long)v);
                }
            }
        }
        const unsigned cm = __ballot_sync(0xffffffffu, claimed);
        if (cm) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&sc.ctr->n_entries, __popc(cm));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (claimed) {
                const int at = base + __popc(cm & ((1u << lane) - 1));
                sc.slist[at] = (int)s;
                sc.sent[at] = hk2;
            }
        }
    }
    const int pmax = __reduce_max_sync(0xffffffffu, probes);
    if (lane == 0 && pmax > 0) atomicMax(&sc.ctr->max_probe, pmax);
}

// ---- per unique (segment, voxel): Eq. 3 term, |V_m|, label at batch start ------
// Per-segment sums gather in shared memory first (one global atomic per
// block and segment).  Each term t (0 <= t <= 2^32 in 2^-32 fixed point)
// adds as its two 16-bit halves in 32-bit shared atomics (64-bit shared
// atomics are slower); a block's half sums stay below 2^31.  lookup = 0: the labels are left to k_lookup, which
// runs once the previous batch's voxels are in (this kernel then reads no
// map state).
__global__ void k_entries(const FrameParams* fps, BatchScratch bs, const MapRefs* refs, int f0, int lookup)
{
    extern __shared__ unsigned char ent_smem[];
    const FrameParams& fp = fps[f0 + blockIdx.y];
    const Scratch sc = bs.frame(f0 + blockIdx.y);
    const VoxelTable vt = refs[fp.map].vt;
    unsigned* s_hi = (unsigned*)ent_smem;             // [M] sum of the terms' high halves (t >> 16)
    unsigned* s_lo = s_hi + max(fp.M, 1);             // [M] sum of their low halves (t & 0xffff)
    int* s_nv = (int*)(s_lo + max(fp.M, 1));          // [M]
    for (int m = threadIdx.x; m < fp.M; m += blockDim.x) {
        s_hi[m] = 0;
        s_lo[m] = 0;
        s_nv[m] = 0;
    }
    __syncthreads();
    const int ne = sc.ctr->n_entries;
    int maxp = 0;
    if (!sc.ctr->err) {
        // whole warps iterate together (lanes past the end idle), so a warp
        // whose 32 entries share one mask adds its sums with one atomic each
        const int lane = threadIdx.x & 31;
        for (int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < ne; i0 += gridDim.x * blockDim.x) {
            const int i = i0 + lane;
            const bool valid = i < ne;
            const unsigned long long hk = valid ? sc.sent[i] : 0ull;
            const int m = (int)(hk >> 54);
            const unsigned long long key = hk & ((1ull << 54) - 1);
            const SegSlot slot = valid ? sc.sslot[sc.slist[i]] : SegSlot{0ull, {0, 0, 0}};
            float N[3] = {__double2float_rn(unfix(slot.n[0], S_VEC)), __double2float_rn(unfix(slot.n[1], S_VEC)),
                          __double2float_rn(unfix(slot.n[2], S_VEC))};
            float l2 = __fadd_rn(__fadd_rn(__fmul_rn(N[0], N[0]), __fmul_rn(N[1], N[1])), __fmul_rn(N[2], N[2]));
            float term = 0.0f;
            if (l2 > 0.0f) {
                float l = __fsqrt_rn(l2);
                float nv[3] = {__fdiv_rn(N[0], l), __fdiv_rn(N[1], l), __fdiv_rn(N[2], l)};
                int k[3];
                unpack_key(key, k);
                float r[3];
#pragma unroll
                for (int a = 0; a < 3; a++)
                    r[a] = __fsub_rn(__fmul_rn(__fadd_rn((float)k[a], 0.5f), fp.voxel), fp.t[a]);
                float rl2 = __fadd_rn(__fadd_rn(__fmul_rn(r[0], r[0]), __fmul_rn(r[1], r[1])), __fmul_rn(r[2], r[2]));
                if (rl2 > 0.0f) {
                    float rl = __fsqrt_rn(rl2);
                    float dot = __fadd_rn(__fadd_rn(__fmul_rn(r[0], nv[0]), __fmul_rn(r[1], nv[1])),
                                          __fmul_rn(r[2], nv[2]));
                    term = __fdiv_rn(-dot, rl);
                    if (!(term > 0.0f)) term = 0.0f;
                }
            }
            const long long tf = fix32f(term, S_VEC);
            unsigned hi = (unsigned)(tf >> 16), lo = (unsigned)(tf & 0xffff);
            const int m0 = __shfl_sync(0xffffffffu, m, 0);
            if (__all_sync(0xffffffffu, valid && m == m0)) {
                hi = __reduce_add_sync(0xffffffffu, hi);
                lo = __reduce_add_sync(0xffffffffu, lo);
                if (lane == 0) {
                    atomicAdd(&s_hi[m0 - 1], hi);
                    atomicAdd(&s_lo[m0 - 1], lo);
                    atomicAdd(&s_nv[m0 - 1], 32);
                }
            } else if (valid) {
                if (hi) atomicAdd(&s_hi[m - 1], hi);
                if (lo) atomicAdd(&s_lo[m - 1], lo);
                atomicAdd(&s_nv[m - 1], 1);
            }
            if (!valid || !lookup) continue;
            // label in the map at the start of the batch (-1: absent then)
            unsigned long long h = mix64(key) & vt.mask;
            int lab = -1, probes = 0;
            while (true) {
                const unsigned long long kk = vt.keys[h];
                if (kk == key) { lab = vt.labels[h]; break; }
                if (kk == EMPTY_KEY) break;
                h = (h + 1) & vt.mask;
                if (++probes > (int)vt.mask) { set_err(sc.ctr, DISC_ERR_TABLE_FULL); break; }
            }
            maxp = max(maxp, probes);
            sc.elab[i] = lab;
        }
    }
    __syncthreads();
    for (int m = threadIdx.x; m < fp.M; m += blockDim.x) {
        if (s_nv[m]) {
            const long long sum = (long long)s_hi[m] * 65536 + (long long)s_lo[m];
            atomicAdd((unsigned long long*)&sc.ang[m], (unsigned long long)sum);
            atomicAdd(&sc.nvox[m], s_nv[m]);
        }
    }
    const int pm = __reduce_max_sync(0xffffffffu, maxp);
    if ((threadIdx.x & 31) == 0 && pm > 0) atomicMax(&sc.ctr->max_probe, pm);
}

// ---- Eq. 2-3: S_angle = mean of the voxel terms; Q per segment -------------------
__global__ void k_quality(const FrameParams* fps, BatchScratch bs)
{
    const FrameParams& fp = fps[blockIdx.x];
    const Scratch sc = bs.frame(blockIdx.x);
    int live = 0;
    for (int m = threadIdx.x; m < fp.M; m += blockDim.x) {
        float* S = sc.S + 5 * m;
        const int nv = sc.nvox[m];
        float sa = 0.0f;
        if (nv > 0) {
            sa = __double2float_rn(__ddiv_rn(unfix(sc.ang[m], S_VEC), (double)nv));
            live++;
        }
        S[1] = sa;
        S[4] = __fmul_rn(__fmul_rn(__fmul_rn(S[0], sa), S[2]), S[3]);
    }
    live = warp_sum(live);
    if ((threadIdx.x & 31) == 0 && live) atomicAdd(&sc.ctr->live_segments, live);
}

// ---- host launchers ------------------------------------------------------------------
int launch_slot_clear(const BatchScratch& bs, int B, int D, int MM, cudaStream_t st)
{
    k_slot_clear<<<dim3(64, B), 256, 0, st>>>(bs, D, MM);
    k_slot_reset<<<(B + 127) / 128, 128, 0, st>>>(bs, B);
    return 2;
}

// launch on frames [f0, f0 + nb) of the batch
int launch_backproject(const FrameParams* fps, const BatchScratch& bs, int f0, int nb, int H, int W, cudaStream_t st)
{
    dim3 b(BP_TX, BP_TY), g((W + BP_TX - 1) / BP_TX, (H + BP_TY - 1) / BP_TY, nb);
    k_backproject<<<g, b, 0, st>>>(fps, bs, f0);
    return 1;
}

int launch_entries(const FrameParams* fps, const BatchScratch& bs, const MapRefs* refs, int f0, int nb, int Mmax,
                   bool lookup, cudaStream_t st)
{
    const size_t smem = 12 * (size_t)std::max(Mmax, 1) + 16;
    k_entries<<<dim3(152 * 2, nb), 256, smem, st>>>(fps, bs, refs, f0, lookup ? 1 : 0);  // 3 x 4 B per mask
    return 1;
}

int launch_quality(const FrameParams* fps, const BatchScratch& bs, int B, cudaStream_t st)
{
    k_quality<<<B, 256, 0, st>>>(fps, bs);
    return 1;
}

}  // namespace disc
