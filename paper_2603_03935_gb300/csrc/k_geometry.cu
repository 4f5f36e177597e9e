// Geometry kernels of the integration step, batched over the frames of a batch
// (they only read the map):
//   Sec. III-A  masked depth -> world points -> voxel keys and pixel normals;
//               per-segment voxel sets V_m in the frame slot's hash
//   Eq. 3       per voxel max(0, -r_v . n_v), summed exactly per segment
//   Sec. III-B  label of every voxel in the map as it stood at the start of
//               the batch (voxels absent then are re-probed by the serial
//               overlap kernel, which sees the inserts of earlier frames)
//   Eq. 2       Q = S_size * S_angle * S_sem * S_dist per segment
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
    const int n = max(ne, max(D, MM));
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < ne) sc.sslot[sc.slist[i]] = SegSlot{0ull, {0, 0, 0}};
        if (i < D) sc.sumF[i] = 0;
        if (i < MM) {
            sc.npix[i] = 0;
            sc.ang[i] = 0;
            sc.nvox[i] = 0;
            sc.segrep[i] = -1;
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

// ---- Sec. III-A: world point of pixel (u, v) at depth z -------------------------
__device__ __forceinline__ void world_point(const FrameParams& fp, int u, int v, float z, float p[3])
{
    float xc = __fdiv_rn(__fmul_rn(__fsub_rn(__fadd_rn((float)u, 0.5f), fp.cx), z), fp.fx);
    float yc = __fdiv_rn(__fmul_rn(__fsub_rn(__fadd_rn((float)v, 0.5f), fp.cy), z), fp.fy);
#pragma unroll
    for (int r = 0; r < 3; r++)
        p[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(fp.R[3 * r], xc), __fmul_rn(fp.R[3 * r + 1], yc)),
                                   __fmul_rn(fp.R[3 * r + 2], z)),
                         fp.t[r]);
}

__device__ __forceinline__ bool pix_valid(const FrameParams& fp, int u, int v, int lab)
{
    if (u < 0 || v < 0 || u >= fp.W || v >= fp.H) return false;
    size_t i = (size_t)v * fp.W + u;
    if (fp.labels[i] != lab) return false;
    float z = fp.depth[i];
    return z >= fp.z_min && z <= fp.z_max;
}

// ---- back-projection + per-segment voxel dedupe (one thread per pixel) ----------
// Block (32, 8): a warp is 32 consecutive pixels of one row; pixel counters are
// aggregated with ballots before one atomic per warp.
__global__ void k_backproject(const FrameParams* fps, BatchScratch bs)
{
    const FrameParams& fp = fps[blockIdx.z];
    const Scratch sc = bs.frame(blockIdx.z);
    if (fp.M <= 0) return;  // uniform per block
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y * blockDim.y + threadIdx.y;
    const bool inside = u < fp.W && v < fp.H;
    int lab = 0;
    float z = 0.0f;
    bool active = inside && !sc.ctr->err;
    if (active) {
        const size_t idx = (size_t)v * fp.W + u;
        lab = fp.labels[idx];
        active = lab >= 1 && lab <= fp.M && sc.npix[lab - 1] >= fp.min_px;
        if (active) {
            z = fp.depth[idx];
            active = z >= fp.z_min && z <= fp.z_max;
        }
    }
    float p0[3] = {0.0f, 0.0f, 0.0f};
    unsigned long long key = 0;
    bool keyed = false;
    if (active) {
        world_point(fp, u, v, z, p0);
        keyed = voxel_key(p0[0], p0[1], p0[2], fp.voxel, &key);
    }
    const unsigned wmask = __activemask();
    const unsigned nvalid = __popc(__ballot_sync(wmask, keyed));
    const unsigned ndrop = __popc(__ballot_sync(wmask, active && !keyed));
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(wmask) - 1;
    if (lane == leader) {
        if (nvalid) atomicAdd(&sc.ctr->valid_pixels, (int)nvalid);
        if (ndrop) atomicAdd(&sc.ctr->dropped_pixels, (int)ndrop);
    }
    // pixel normal (zero when it has none)
    long long nfix[3] = {0, 0, 0};
    if (keyed) {
        // image-space tangents: forward differences, backward at the mask's edge
        int ua = -1, ub = -1, va = -1, vb = -1;
        if (pix_valid(fp, u + 1, v, lab)) { ua = u + 1; ub = u; }
        else if (pix_valid(fp, u - 1, v, lab)) { ua = u; ub = u - 1; }
        if (pix_valid(fp, u, v + 1, lab)) { va = v + 1; vb = v; }
        else if (pix_valid(fp, u, v - 1, lab)) { va = v; vb = v - 1; }
        if (ua >= 0 && va >= 0) {
            float pa[3], pb[3], qa[3], qb[3];
            world_point(fp, ua, v, fp.depth[(size_t)v * fp.W + ua], pa);
            world_point(fp, ub, v, fp.depth[(size_t)v * fp.W + ub], pb);
            world_point(fp, u, va, fp.depth[(size_t)va * fp.W + u], qa);
            world_point(fp, u, vb, fp.depth[(size_t)vb * fp.W + u], qb);
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
                float l = __fsqrt_rn(l2);
#pragma unroll
                for (int r = 0; r < 3; r++) n[r] = __fdiv_rn(n[r], l);
                // orient toward the camera
                float vd = __fadd_rn(__fadd_rn(__fmul_rn(__fsub_rn(p0[0], fp.t[0]), n[0]),
                                               __fmul_rn(__fsub_rn(p0[1], fp.t[1]), n[1])),
                                     __fmul_rn(__fsub_rn(p0[2], fp.t[2]), n[2]));
                if (vd > 0.0f) {
#pragma unroll
                    for (int r = 0; r < 3; r++) n[r] = -n[r];
                }
#pragma unroll
                for (int r = 0; r < 3; r++) nfix[r] = fix32f(n[r], S_VEC);
            }
        }
    }

    // Runs of consecutive lanes with the same (mask, voxel) key: a segmented
    // inclusive scan gives the last lane of each run the run's exact normal
    // sums; that lane alone updates the hash.  A key that reappears later in
    // the warp forms a second run (a second, still exact, update).
    const unsigned long long hk = keyed ? (((unsigned long long)lab << 54) | key) : 0ull;
    const unsigned long long hk_prev = __shfl_up_sync(wmask, hk, 1);
    const unsigned long long hk_next = __shfl_down_sync(wmask, hk, 1);
    const bool head = lane == 0 || hk_prev != hk;
    const bool tail = lane == 31 || hk_next != hk;
    const unsigned heads = __ballot_sync(wmask, head);
    const int run_start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        long long o0 = __shfl_up_sync(wmask, nfix[0], d);
        long long o1 = __shfl_up_sync(wmask, nfix[1], d);
        long long o2 = __shfl_up_sync(wmask, nfix[2], d);
        if (lane - d >= run_start) {
            nfix[0] += o0;
            nfix[1] += o1;
            nfix[2] += o2;
        }
    }
    int probes = 0;
    if (keyed && tail) {
        // insert (mask, voxel) into the slot's hash; the winner of an empty
        // slot appends it to the entry list
        unsigned long long s = mix64(hk) & sc.smask;
        bool ok = true;
        while (true) {
            const unsigned long long cur = sc.sslot[s].key;
            if (cur == hk) break;
            if (cur == 0ull) {
                const unsigned long long prev = atomicCAS(&sc.sslot[s].key, 0ull, hk);
                if (prev == 0ull) {
                    const int at = atomicAdd(&sc.ctr->n_entries, 1);
                    sc.slist[at] = (int)s;
                    sc.sent[at] = hk;
                    break;
                }
                if (prev == hk) break;
            }
            s = (s + 1) & sc.smask;
            if (++probes > (int)sc.smask) {
                set_err(sc.ctr, DISC_ERR_TABLE_FULL);
                ok = false;
                break;
            }
        }
        if (ok) {
            SegSlot& slot = sc.sslot[s];
            if (nfix[0]) atomicAdd((unsigned long long*)&slot.n[0], (unsigned long long)nfix[0]);
            if (nfix[1]) atomicAdd((unsigned long long*)&slot.n[1], (unsigned long long)nfix[1]);
            if (nfix[2]) atomicAdd((unsigned long long*)&slot.n[2], (unsigned long long)nfix[2]);
        }
    }
    const int pmax = __reduce_max_sync(wmask, probes);
    if (lane == leader && pmax > 0) atomicMax(&sc.ctr->max_probe, pmax);
}

// ---- per unique (segment, voxel): Eq. 3 term, |V_m|, label at batch start ------
// Per-segment sums gather in shared memory first (one global atomic per
// block and segment).
__global__ void k_entries(const FrameParams* fps, BatchScratch bs, VoxelTable vt)
{
    extern __shared__ unsigned char ent_smem[];
    const FrameParams& fp = fps[blockIdx.y];
    const Scratch sc = bs.frame(blockIdx.y);
    long long* s_ang = (long long*)ent_smem;         // [M]
    int* s_nv = (int*)(s_ang + max(fp.M, 1));         // [M]
    for (int m = threadIdx.x; m < fp.M; m += blockDim.x) {
        s_ang[m] = 0;
        s_nv[m] = 0;
    }
    __syncthreads();
    const int ne = sc.ctr->n_entries;
    int maxp = 0;
    if (!sc.ctr->err) {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += gridDim.x * blockDim.x) {
            const unsigned long long hk = sc.sent[i];
            const int m = (int)(hk >> 54);
            const unsigned long long key = hk & ((1ull << 54) - 1);
            const SegSlot slot = sc.sslot[sc.slist[i]];
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
            atomicAdd((unsigned long long*)&s_ang[m - 1], (unsigned long long)fix32f(term, S_VEC));
            atomicAdd(&s_nv[m - 1], 1);
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
            atomicAdd((unsigned long long*)&sc.ang[m], (unsigned long long)s_ang[m]);
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

int launch_backproject(const FrameParams* fps, const BatchScratch& bs, int B, int H, int W, cudaStream_t st)
{
    dim3 b(32, 8), g((W + 31) / 32, (H + 7) / 8, B);
    k_backproject<<<g, b, 0, st>>>(fps, bs);
    return 1;
}

int launch_entries(const FrameParams* fps, const BatchScratch& bs, const VoxelTable& vt, int B, int Mmax,
                   cudaStream_t st)
{
    const size_t smem = 12 * (size_t)std::max(Mmax, 1) + 16;
    k_entries<<<dim3(152 * 2, B), 256, smem, st>>>(fps, bs, vt);
    k_quality<<<B, 256, 0, st>>>(fps, bs);
    return 2;
}

}  // namespace disc
