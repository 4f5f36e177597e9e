// Sec. III-A: the points of each segment are filtered by DBSCAN before they
// are voxelised.  A point (pixel of an active mask with valid depth and an
// in-range voxel) is core when at least min_pts points of its segment, itself
// included, lie within eps -- ((dx*dx + dy*dy) + dz*dz) <= eps*eps in fp32 --
// and kept when it is core or within eps of a core point; the other points
// are noise and count as invalid depth for the back-projection.
//
// Per frame (chunks of frames like the back-projection):
//   k_db_points   world point of every point pixel; its (mask, cell) in a
//                 hash of cells 1.001 eps wide, so every point within eps of
//                 a point lies in the 27 cells around it
//   k_db_offsets  first position of every cell in the cell-ordered list
//   k_db_scatter  the points in cell order
//   k_db_core     core flags (counting stops at min_pts)
//   k_db_noise    noise flags of the points with no core point within eps
#include "disc_common.cuh"
#include "kernels.h"

namespace disc {

namespace {

__device__ __forceinline__ void db_err(const Scratch& sc, int code) { atomicCAS(&sc.ctr->err, 0, code); }

__device__ __forceinline__ unsigned long long cell_key(int lab, int cx, int cy, int cz)
{
    return ((unsigned long long)lab << 54) | ((unsigned long long)(cx + KEY_BIAS) << (2 * KEY_BITS)) |
           ((unsigned long long)(cy + KEY_BIAS) << KEY_BITS) | (unsigned long long)(cz + KEY_BIAS);
}

__device__ __forceinline__ void cell_of(const FrameParams& fp, float4 p, int c[3])
{
    c[0] = (int)floorf(__fmul_rn(p.x, fp.db_inv_cell));
    c[1] = (int)floorf(__fmul_rn(p.y, fp.db_inv_cell));
    c[2] = (int)floorf(__fmul_rn(p.z, fp.db_inv_cell));
}

// hash slot of a cell, or -1
__device__ __forceinline__ long long find_cell(const Scratch& sc, unsigned long long key)
{
    unsigned long long h = mix64(key) & sc.smask;
    for (unsigned long long pr = 0; pr <= sc.smask; pr++) {
        const unsigned long long cur = sc.dkey[h];
        if (cur == key) return (long long)h;
        if (cur == 0ull) return -1;
        h = (h + 1) & sc.smask;
    }
    return -1;
}

__device__ __forceinline__ bool within(float4 a, float4 b, float eps2)
{
    const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)) <= eps2;
}

// Visit the points of the 27 cells around point p (same mask) that lie
// within eps; f returns false to stop.
template <class F>
__device__ __forceinline__ void for_neighbours(const FrameParams& fp, const Scratch& sc, float4 p, F&& f)
{
    int c[3];
    cell_of(fp, p, c);
    const int lab = __float_as_int(p.w);
    for (int dx = -1; dx <= 1; dx++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dz = -1; dz <= 1; dz++) {
                const int q[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
                if (q[0] < -KEY_BIAS || q[0] > KEY_BIAS - 1 || q[1] < -KEY_BIAS || q[1] > KEY_BIAS - 1 ||
                    q[2] < -KEY_BIAS || q[2] > KEY_BIAS - 1)
                    continue;
                const long long h = find_cell(sc, cell_key(lab, q[0], q[1], q[2]));
                if (h < 0) continue;
                const int s0 = sc.dstart[sc.dpos[h]], n = sc.dcnt[h];
                for (int j = 0; j < n; j++) {
                    const int o = sc.dorder[s0 + j];
                    if (within(p, sc.dpt[o], fp.db_eps2) && !f(o)) return;
                }
            }
}

}  // namespace

// one thread per pixel of frames [f0, f0 + gridDim.y)
__global__ void k_db_points(const FrameParams* fps, BatchScratch bs, int f0)
{
    const FrameParams& fp = fps[f0 + blockIdx.y];
    const Scratch sc = bs.frame(f0 + blockIdx.y);
    if (fp.db_min_pts <= 0 || fp.M <= 0 || sc.ctr->err) return;  // uniform per block
    const int npx = fp.W * fp.H;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool pt = false;
    float p[3] = {0.0f, 0.0f, 0.0f};
    int lab = 0;
    if (idx < npx) {
        const int u = idx % fp.W, v = idx / fp.W;
        lab = fp.labels[idx];
        const float z = fp.depth[idx];
        if (lab >= 1 && lab <= fp.M && sc.npix[lab - 1] >= fp.min_px && z >= fp.z_min && z <= fp.z_max) {
            world_point(fp, u, v, z, p);
            unsigned long long vk;
            pt = voxel_key(p[0], p[1], p[2], fp.inv_voxel, &vk);
        }
        sc.dflag[idx] = 0;
        sc.dpt[idx] = make_float4(p[0], p[1], p[2], __int_as_float(lab));
    }
    // the pixels of a warp that share a cell claim it once
    unsigned long long key = 0ull;
    if (pt) {
        int c[3];
        cell_of(fp, make_float4(p[0], p[1], p[2], 0.0f), c);
        key = cell_key(lab, c[0], c[1], c[2]);
    }
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    long long h = -1;
    if (pt && lane == __ffs(grp) - 1) {
        unsigned long long s = mix64(key) & sc.smask;
        for (unsigned long long pr = 0;; pr++) {
            const unsigned long long cur = sc.dkey[s];
            if (cur == key) break;
            if (cur == 0ull) {
                const unsigned long long prev = atomicCAS(&sc.dkey[s], 0ull, key);
                if (prev == 0ull) {
                    const int at = atomicAdd(&sc.ctr->n_cells, 1);
                    sc.dlist[at] = (int)s;
                    sc.dpos[s] = at;
                    break;
                }
                if (prev == key) break;
            }
            s = (s + 1) & sc.smask;
            if (pr > sc.smask) {
                db_err(sc, DISC_ERR_TABLE_FULL);
                s = ~0ull;
                break;
            }
        }
        if (s != ~0ull) {
            h = (long long)s;
            atomicAdd(&sc.dcnt[s], __popc(grp));
        }
    }
    if (pt) h = __shfl_sync(grp, h, __ffs(grp) - 1);
    if (idx < npx) sc.dcell[idx] = pt ? (int)h : -1;
}

// one block per frame: exclusive scan of the cell sizes in list order
__global__ void k_db_offsets(const FrameParams* fps, BatchScratch bs, int f0)
{
    const FrameParams& fp = fps[f0 + blockIdx.x];
    const Scratch sc = bs.frame(f0 + blockIdx.x);
    if (fp.db_min_pts <= 0 || fp.M <= 0 || sc.ctr->err) return;
    __shared__ int wsum[32];
    __shared__ int carry;
    const int n = sc.ctr->n_cells;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const int x = i < n ? sc.dcnt[sc.dlist[i]] : 0;
        int incl = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int nw = blockDim.x >> 5;
            int w = lane < nw ? wsum[lane] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += y;
            }
            if (lane < nw) wsum[lane] = w;  // inclusive warp totals
        }
        __syncthreads();
        const int before = carry + (warp > 0 ? wsum[warp - 1] : 0) + incl - x;
        if (i < n) {
            sc.dstart[i] = before;
            sc.dfill[i] = 0;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + x;
        __syncthreads();
    }
}

__global__ void k_db_scatter(const FrameParams* fps, BatchScratch bs, int f0)
{
    const FrameParams& fp = fps[f0 + blockIdx.y];
    const Scratch sc = bs.frame(f0 + blockIdx.y);
    if (fp.db_min_pts <= 0 || fp.M <= 0 || sc.ctr->err) return;
    const int npx = fp.W * fp.H;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int h = idx < npx ? sc.dcell[idx] : -1;
    const unsigned grp = __match_any_sync(0xffffffffu, h);
    if (h < 0) return;
    const int lp = sc.dpos[h];
    int base = 0;
    const int lead = __ffs(grp) - 1;
    if (lane == lead) base = atomicAdd(&sc.dfill[lp], __popc(grp));
    base = __shfl_sync(grp, base, lead);
    sc.dorder[sc.dstart[lp] + base + __popc(grp & ((1u << lane) - 1))] = idx;
}

__global__ void k_db_core(const FrameParams* fps, BatchScratch bs, int f0)
{
    const FrameParams& fp = fps[f0 + blockIdx.y];
    const Scratch sc = bs.frame(f0 + blockIdx.y);
    if (fp.db_min_pts <= 0 || fp.M <= 0 || sc.ctr->err) return;
    const int npx = fp.W * fp.H;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= npx || sc.dcell[idx] < 0) return;
    const float4 p = sc.dpt[idx];
    int cnt = 0;
    const int need = fp.db_min_pts;
    for_neighbours(fp, sc, p, [&](int) { return ++cnt < need; });
    if (cnt >= need) sc.dflag[idx] = 1;
}

__global__ void k_db_noise(const FrameParams* fps, BatchScratch bs, int f0)
{
    const FrameParams& fp = fps[f0 + blockIdx.y];
    const Scratch sc = bs.frame(f0 + blockIdx.y);
    if (fp.db_min_pts <= 0 || fp.M <= 0 || sc.ctr->err) return;
    const int npx = fp.W * fp.H;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    bool noise = false;
    if (idx < npx && sc.dcell[idx] >= 0 && !(sc.dflag[idx] & 1)) {
        bool near_core = false;
        for_neighbours(fp, sc, sc.dpt[idx], [&](int o) {
            near_core = (sc.dflag[o] & 1) != 0;
            return !near_core;
        });
        if (!near_core) {
            sc.dflag[idx] = 2;
            noise = true;
        }
    }
    const int nn = __popc(__ballot_sync(0xffffffffu, noise));
    if ((threadIdx.x & 31) == 0 && nn) atomicAdd(&sc.ctr->denoised, nn);
}

int launch_dbscan(const FrameParams* fps, const BatchScratch& bs, int f0, int nb, int H, int W, cudaStream_t st)
{
    const int npx = H * W;
    dim3 g((npx + 255) / 256, nb);
    k_db_points<<<g, 256, 0, st>>>(fps, bs, f0);
    k_db_offsets<<<nb, 1024, 0, st>>>(fps, bs, f0);
    k_db_scatter<<<g, 256, 0, st>>>(fps, bs, f0);
    k_db_core<<<g, 256, 0, st>>>(fps, bs, f0);
    k_db_noise<<<g, 256, 0, st>>>(fps, bs, f0);
    return 5;
}

}  // namespace disc
